"""Benchmark: interval-SVD solves/s at residual <= 1e-10 on one GB300.

Workload (default): the known-spectrum sparse matrix of 200000 x 100000 made of
25000 dense 8 x 4 N(0,1) blocks with random row and column permutations
(seed 2), interior interval holding 200 singular values near the median
(endpoints at gap midpoints), N = 32, L = 32, M = 8, ell = 2, V_in N(0,1)
(seed 3). One step = one complete cmsvd_solve_interval (all of Alg. 1: shifted
solves, moments, truncation, QR, Rayleigh-Ritz, residuals). A step counts only
if it returns all 200 triplets with residual <= 1e-10.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

Secondary keys of the same line: the 2e6 x 1e6 mixed-precision workload (banded plus
random columns, 32M nonzeros, Krylov solver) in mixed precision and in FP64
(c3_mixed_vs_fp64: one timed solve each, about 70 s), the full-scale SpMM roofline
(spmm_roofline), the 2000 x 1000 Krylov workload in both precisions (krylov_workload),
64 batched problems (batched_workload) and the serving loop (serving_workload).

value: device-resident inputs (the matrix and V_in stay in HBM), CUDA events
around each call on the caller's stream, L2 flushed (256 MiB write) between
steps outside the timed window. e2e: the same through the C ABI with V_in in
pinned host memory and all triplets copied back to pinned host memory inside
the timed window. Multi-GPU: independent replicas (the method needs no
exchange between GPUs), max time over ranks. --impl reference times the CPU
oracle (NumPy FP64 direct solves) on the same workload on rank 0: W untimed and K
timed full solves, about 6 s each on 16 host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2109_13655_gb300 import synth  # noqa: E402

METRIC = "interval-SVD solves/s at residual<=1e-10, mixed vs FP64 on 1 GB300; p50/p99 latency"
UNIT = "solves/s"


# ----------------------------------------------------------------------------- workloads
def workload(name: str):
    if name == "block_permuted_200000x100000":
        bp = synth.block_permuted(25000, 8, 4, seed=2)
        s = bp.sigmas_desc()
        a, b, f = synth.window_interval(s, 50000, 200, min_rel_gap=1e-6, max_shift=10)
        cfg = dict(N=32, L=32, M=8, ell=2)
        return dict(name=name, A=bp.A, a=a, b=b, t=200, norm_A=float(s[0]), cfg=cfg, seed=3,
                    desc="200000x100000 CSR, 25000 permuted 8x4 N(0,1) blocks (nnz 800000), "
                         "200 interior sigma, N=32 L=32 M=8 ell=2")
    if name == "random_sparse_2000x1000":
        A = synth.random_sparse(2000, 1000, 8, seed=0)
        s = np.linalg.svd(A.to_dense(), compute_uv=False)
        a, b, _ = synth.window_interval(s, 400, 20)
        cfg = dict(N=16, L=16, M=4, ell=1)
        return dict(name=name, A=A, a=a, b=b, t=20, norm_A=float(s[0]), cfg=cfg, seed=1,
                    desc="2000x1000 CSR, 8 nnz/row N(0,1), sigma ranked 400-419, N=16 L=16 M=4")
    if name == "banded_random_2000000x1000000":
        g = np.loadtxt(os.path.join(ROOT, "tests", "golden", "banded_random_2000000x1000000_top.txt"))
        t = 85
        cfg = dict(N=32, L=32, M=8, ell=2, alpha=0.2)
        return dict(name=name, A=synth.banded_random(), a=0.5 * (g[t - 1] + g[t]), b=1.01 * g[0], t=t,
                    norm_A=float(g[0]), cfg=cfg, seed=11, golden=g[:t],
                    desc="2000000x1000000 CSR, 16 nnz/row (8 within +-5000 of the diagonal position, 8 uniform), "
                         "U(-1,1) bf16-exact values (nnz 32M); exterior window of the 85 largest sigma (a at the "
                         "widest relative gap near the 100th value, b = 1.01 sigma_1); N=32 L=32 M=8 ell=2 "
                         "alpha=0.2; Krylov solver")
    raise ValueError(name)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- reference arm (CPU oracle)
def run_reference(args, w, rank):
    if rank != 0:
        return
    from oracle import cmsvd_oracle as O
    A, cfg = w["A"], w["cfg"]
    Vin = synth.gaussian_block(A.n, cfg["L"], w["seed"])
    solver = O.ShiftedSolver(A)
    times, ok = [], True
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = O.solve_interval(A, w["a"], w["b"], cfg["N"], cfg["L"], cfg["M"], Vin, ell=cfg["ell"],
                             norm_A=w["norm_A"], solver=solver)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            ok &= r.sigma.size == w["t"] and float(np.max(r.res_u)) <= 1e-10
    v = len(times) / sum(times)
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": w["desc"], **cfg},
            "all_steps_valid": bool(ok),
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{len(times)} full oracle solves of the workload (NumPy/OpenBLAS FP64; "
                                       f"dense steps on OpenBLAS's default {cores} threads, the stacked "
                                       f"per-component solves on one thread)"}}
    print(json.dumps(line), flush=True)


def cpu_baseline(w, budget_s=30.0):
    """The oracle as it stands, timed on this host: full solves of the workload until ~budget_s."""
    from oracle import cmsvd_oracle as O
    A, cfg = w["A"], w["cfg"]
    Vin = synth.gaussian_block(A.n, cfg["L"], w["seed"])
    solver = O.ShiftedSolver(A)
    times = []
    t_start = time.perf_counter()
    while not times or (time.perf_counter() - t_start < budget_s * 0.5 and len(times) < 3):
        t0 = time.perf_counter()
        O.solve_interval(A, w["a"], w["b"], cfg["N"], cfg["L"], cfg["M"], Vin, ell=cfg["ell"], norm_A=w["norm_A"],
                         solver=solver)
        times.append(time.perf_counter() - t0)
    cores = os.cpu_count()
    return {"value": len(times) / sum(times), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(times)} full oracle solve(s) of the same workload, {sum(times):.1f} s total; "
                      f"dense steps on OpenBLAS's default {cores} threads, the stacked per-component "
                      f"solves on one thread"}


# ----------------------------------------------------------------------------- our arm
def run_ours(args, w, rank, world, local_rank):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2109_13655_gb300 import binding as B

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank)
    A, cfg = w["A"], w["cfg"]
    ctx = B.Context()
    M = B.Matrix.from_csr(ctx, A)
    p = B.params(N=cfg["N"], L=cfg["L"], M=cfg["M"], ell=cfg["ell"], norm_A=w["norm_A"], profile=1)
    Vin_h = synth.gaussian_block(A.n, cfg["L"], w["seed"])
    Vin = torch.from_numpy(Vin_h).to(dev)
    ws = M.workspace(p)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def one(Vd):
        status, r = B.cmsvd_solve_interval(M.handle, w["a"], w["b"], p, Vd, ws)
        return status, r

    def check(r):
        st = B.cmsvd_result_stats(r)
        t = B.cmsvd_result_count(r)
        return st, t == w["t"] and st["max_res_u"] <= 1e-10 and st["max_res_v"] <= 1e-10

    setup_ms = None
    for k in range(args.warmup):
        _, r = one(Vin)
        if k == 0:   # the first solve on a matrix builds the components of A^T A (solver AUTO), on the host
            setup_ms = B.cmsvd_result_stats(r)["ms_components"]
        B.cmsvd_result_destroy(r)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats, valid, launches = [], True, 0
    with ClockSampler(local_rank) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            _, r = one(Vin)
            ev[k][1].record(stream)
            st, ok = check(r)
            valid &= ok
            stats.append(st)
            launches += st["kernel_launches"]
            B.cmsvd_result_destroy(r)
        torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(ms) / 1e3
    # ---- e2e through the C ABI with host buffers
    Vin_pin = torch.from_numpy(Vin_h).pin_memory()
    Vd = torch.empty_like(Vin)
    t_out = w["t"]
    outs = [torch.empty(n, dtype=torch.float64).pin_memory() for n in
            (t_out, A.m * t_out, A.n * t_out, t_out, t_out, t_out)]
    h2d = Vin_pin.numel() * 8
    d2h = sum(o.numel() * 8 for o in outs)
    e2e_ms = []
    for k in range(max(1, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Vd.copy_(Vin_pin, non_blocking=True)
        _, r = one(Vd)
        B.cmsvd_result_copy(r, *outs)
        B.cmsvd_result_destroy(r)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    # ---- max over ranks
    tmax, e2e_max = max_over_ranks([total_s, sum(e2e_ms) / len(e2e_ms)], dist, dev)
    krylov = measure_krylov(B, ctx, dev) if (rank == 0 and args.krylov) else None
    table2 = measure_table2(B, dev) if (rank == 0 and args.table2) else None
    batched = measure_batched(B, dev) if (rank == 0 and args.batched) else None
    serving = measure_serving(B) if (rank == 0 and args.serving) else None
    spmm_big = measure_spmm(B, dev) if (rank == 0 and args.spmm) else None
    c3 = measure_c3(B, dev) if (rank == 0 and args.c3) else None
    if rank == 0:
        value = job_throughput(args.steps, world, tmax)
        prof = aggregate_profile(stats)
        dom = max(prof, key=lambda k: prof[k]["ms"]) if prof else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tmax / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": w["desc"], **cfg, "t": w["t"],
                       "solver": {0: "auto", 1: "krylov", 2: "direct", 3: "dense"}[stats[-1]["solver_used"]],
                       "l2": "flushed (256 MiB write) before every step, outside the timed window",
                       "parallelism": f"replicas x{world}"},
            "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)),
                           "min": float(np.min(ms))},
            "all_steps_valid": bool(valid),
            "setup_ms_outside_timing": {"components_of_AtA": setup_ms},
            "phase_ms": {k: float(np.median([s[k] for s in stats])) for k in
                         ("ms_solve", "ms_truncate", "ms_qr", "ms_ritz")},
            "clocks": clk.summary(),
            "e2e": {"value": world / (e2e_max / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "kernel_profile": prof,
            "roofline": roofline(dom, prof, stats, w) if dom else None,
            "precision_note": "the direct solver used on this workload is exact; CMSVD_MIXED changes only the "
                              "Krylov solver, measured below",
            "krylov_workload": krylov,
        }
        if table2 is not None:
            line["exp3_table2"] = table2
        if batched is not None:
            line["batched_workload"] = batched
        if serving is not None:
            line["serving_workload"] = serving
        if spmm_big is not None:
            line["spmm_roofline"] = spmm_big
        if c3 is not None:
            line["c3_mixed_vs_fp64"] = c3
        if args.cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w)
        print(json.dumps(line), flush=True)
    M.close()
    ctx.close()
    if dist:
        dist.destroy_process_group()


def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise maximum of per-rank timings (replicas: the slowest rank sets the job time)."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def job_throughput(steps_per_rank: int, world: int, max_seconds: float) -> float:
    """Whole-job solves/s: every rank runs steps_per_rank independent solves (weak scaling)."""
    return world * steps_per_rank / max_seconds


def measure_krylov(B, ctx, dev, steps=3):
    """The 2000 x 1000 random sparse workload (Krylov solver): FP64 vs mixed, device-resident
    inputs, CUDA events around each call, every step checked (20 triplets, residual <= 1e-10)."""
    import torch
    w = workload("random_sparse_2000x1000")
    A, cfg = w["A"], w["cfg"]
    M = B.Matrix.from_csr(ctx, A)
    Vin = torch.from_numpy(synth.gaussian_block(A.n, cfg["L"], w["seed"])).to(dev)
    out = {"description": w["desc"]}
    for name, prec in (("fp64", B.FP64), ("mixed", B.MIXED)):
        p = B.params(N=cfg["N"], L=cfg["L"], M=cfg["M"], ell=cfg["ell"], norm_A=w["norm_A"], solver="krylov",
                     precision=prec)
        ws = M.workspace(p)
        ms, ok, st = [], True, None
        for k in range(steps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, r = B.cmsvd_solve_interval(M.handle, w["a"], w["b"], p, Vin, ws)
            e1.record()
            st = B.cmsvd_result_stats(r)
            t = B.cmsvd_result_count(r)
            B.cmsvd_result_destroy(r)
            torch.cuda.synchronize()
            if k > 0:
                ms.append(e0.elapsed_time(e1))
                ok &= t == w["t"] and st["max_res_u"] <= 1e-10
        out[name] = {"solves_per_s": 1e3 / float(np.mean(ms)), "ms_per_solve": float(np.mean(ms)),
                     "all_steps_valid": bool(ok), "lanczos_steps": int(st["krylov_iters"]),
                     "refine_rounds": int(st["refine_rounds"]), "ms_solve": st["ms_solve"],
                     "ms_rayleigh_ritz": st["ms_truncate"] + st["ms_qr"] + st["ms_ritz"]}
        del ws
    M.close()
    return out


def measure_c3(B, dev):
    """The 2e6 x 1e6 mixed-precision workload (banded plus random columns, 32M nonzeros) through
    the Krylov solver: mixed precision (double-float Lanczos on the FP32 pipe, bf16 storage of A)
    against plain FP64 (FP64 storage), each as one warm-up solve cut short at 96 Lanczos steps
    per pass (it runs the SpMM autotuner and the graph captures) and one timed full solve (CUDA
    events on the caller's stream; the 129 MB L2 is far smaller than the inputs: A and A^T take
    0.4-0.8 GB, every Lanczos block 256 MB). Each solve must return all 85 values with
    residuals <= 1e-10 and sigma within 1e-10 of the expected values (ARPACK, tests/golden).
    Reports per precision: solves/s, Lanczos steps, phase times, kernel classes, the SpMM
    autotuner's picks; and per triplet the mixed-vs-FP64 differences of sigma and residuals."""
    import torch
    w = workload("banded_random_2000000x1000000")
    A, cfg = w["A"], w["cfg"]
    ctx = B.Context()
    Vin = torch.from_numpy(synth.gaussian_block(A.n, cfg["L"], w["seed"])).to(dev)
    out = {"description": w["desc"], "interval": [w["a"], w["b"]], "t": w["t"]}
    res = {}
    for name, prec, storage in (("mixed", B.MIXED, "bf16"), ("fp64", B.FP64, "fp64")):
        M = B.Matrix.from_csr(ctx, A, storage=storage)
        p = B.params(N=cfg["N"], L=cfg["L"], M=cfg["M"], ell=cfg["ell"], alpha=cfg["alpha"], solver="krylov",
                     precision=prec, norm_A=w["norm_A"], profile=1)
        ws = M.workspace(p)
        pw = B.params(N=cfg["N"], L=cfg["L"], M=cfg["M"], ell=1, alpha=cfg["alpha"], solver="krylov",
                      precision=prec, norm_A=w["norm_A"], max_iter=96)
        _, r = B.cmsvd_solve_interval(M.handle, w["a"], w["b"], pw, Vin, ws)          # warm-up
        B.cmsvd_result_destroy(r)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.current_stream()
        e0.record(stream)
        status, r = B.cmsvd_solve_interval(M.handle, w["a"], w["b"], p, Vin, ws)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        t = B.cmsvd_result_count(r)
        st = B.cmsvd_result_stats(r)
        sig, ru, rv = np.zeros(t), np.zeros(t), np.zeros(t)
        B.cmsvd_result_copy(r, sig, None, None, ru, rv)
        B.cmsvd_result_destroy(r)
        truth = np.sort(w["golden"])
        ok = t == w["t"] and float(max(ru.max(), rv.max())) <= 1e-10 and \
            float(np.max(np.abs(sig - truth) / truth)) <= 1e-10
        res[name] = (sig, ru, rv)
        tun = {"A": B.cmsvd_spmm_tuning(M.handle, False, 2 if name == "mixed" else 0, cfg["L"]),
               "At": B.cmsvd_spmm_tuning(M.handle, True, 2 if name == "mixed" else 0, cfg["L"])}
        prof = {B.PROFILE_CLASSES[i]: {"ms": st["prof_ms"][i], "launches": st["prof_launches"][i],
                                       "bytes": st["prof_bytes"][i], "flops": st["prof_flops"][i]}
                for i in range(len(B.PROFILE_CLASSES)) if st["prof_launches"][i]}
        out[name] = {"solves_per_s": 1e3 / ms, "ms_per_solve": ms, "status": int(status), "found": int(t),
                     "all_valid": bool(ok), "lanczos_steps_last_filter": int(st["krylov_iters"]),
                     "max_sigma_rel_err_vs_expected": float(np.max(np.abs(sig - truth) / truth)) if t == w["t"] else None,
                     "max_res_u": float(ru.max()) if t else None, "max_res_v": float(rv.max()) if t else None,
                     "rank": int(st["rank"]), "kernel_launches": int(st["kernel_launches"]),
                     "phase_ms": {k: st[k] for k in ("ms_solve", "ms_truncate", "ms_qr", "ms_ritz")},
                     "kernel_profile": prof, "spmm_autotune": tun,
                     "storage": storage}
        M.close()
        del ws
        torch.cuda.empty_cache()
    ctx.close()
    if res["mixed"][0].size == res["fp64"][0].size and res["fp64"][0].size:
        sm, rm, _ = res["mixed"]
        sf, rf, _ = res["fp64"]
        out["mixed_vs_fp64"] = {"speedup": out["mixed"]["solves_per_s"] / out["fp64"]["solves_per_s"],
                                "max_sigma_rel_diff": float(np.max(np.abs(sm - sf) / sf)),
                                "max_res_u_mixed": float(rm.max()), "max_res_u_fp64": float(rf.max()),
                                "per_triplet_sigma_rel_diff": [float(x) for x in np.abs(sm - sf) / sf],
                                "per_triplet_res_u": {"mixed": [float(x) for x in rm], "fp64": [float(x) for x in rf]}}
    return out


def measure_batched(B, dev, contexts=8, reps=2):
    """64 independent block-permuted problems (10 x 4 blocks, n log-uniform in [2000, 80000],
    m = 2.5 n, N and L in {16, 32}, M = 4, half exterior, half interior, t = floor(L M / 3)):
    one after another from one host thread, against one cmsvd_solve_batch call over
    `contexts` streams. Device-resident inputs; every solve must return its t triplets with
    residuals <= 1e-10."""
    import torch
    probs = synth.batched_problems(64, seed=4)
    ctxs = [B.Context(torch.cuda.Stream()) for _ in range(contexts)]
    mats = [B.Matrix.from_csr(ctxs[i % contexts], p["A"]) for i, p in enumerate(probs)]
    prms = [B.params(N=p["N"], L=p["L"], M=p["M"], norm_A=float(p["sigma"][0])) for p in probs]
    Vs = [torch.from_numpy(synth.gaussian_block(p["A"].n, p["L"], p["seed_v"])).to(dev) for p in probs]
    wss = [M.workspace(q) for M, q in zip(mats, prms)]
    handles = [M.handle for M in mats]
    torch.cuda.synchronize()

    def check(rs):
        ok = True
        for r, p in zip(rs, probs):
            st = B.cmsvd_result_stats(r)
            ok &= B.cmsvd_result_count(r) == p["t"] and st["max_res_u"] <= 1e-10 and st["max_res_v"] <= 1e-10
            B.cmsvd_result_destroy(r)
        return bool(ok)

    def sequential():
        rs = []
        for i in range(len(probs)):
            _, r = B.cmsvd_solve_interval(handles[i], probs[i]["a"], probs[i]["b"], prms[i], Vs[i], wss[i])
            rs.append(r)
        torch.cuda.synchronize()
        return rs

    def batched():
        _, rs = B.cmsvd_solve_batch(handles, [p["a"] for p in probs], [p["b"] for p in probs], prms, Vs, wss)
        torch.cuda.synchronize()
        return rs

    out = {}
    for name, fn in (("sequential", sequential), ("batched", batched)):
        valid = check(fn())                       # warm-up pass
        times = []
        for _ in range(reps):
            t0 = time.perf_counter()
            rs = fn()
            times.append(time.perf_counter() - t0)
            valid &= check(rs)
        best = min(times)
        out[name] = {"solves_per_s": len(probs) / best, "s_per_batch": best, "all_valid": valid}
    for M in mats:
        M.close()
    for c in ctxs:
        c.close()
    out["speedup"] = out["batched"]["solves_per_s"] / out["sequential"]["solves_per_s"]
    out["description"] = (f"64 block-permuted problems (10x4 N(0,1) blocks, n in [2000, 80000] log-uniform, "
                          f"sum n = {sum(p['A'].n for p in probs)}), N,L in {{16,32}}, M=4, half exterior/half "
                          f"interior, t = floor(LM/3); batched = one cmsvd_solve_batch call over {contexts} "
                          f"contexts (streams, one host thread each); wall clock, inputs resident")
    return out


def measure_serving(B, slots=8, rate=200.0, count=300, seed=5):
    """Serving with continuous batching (cmsvd_server_*): 16 resident matrices with rows
    log-uniform in [1e4, 2e5] and c in {8, 16, 32} nonzeros per row, realized as permuted
    2c x c blocks of U(-1,1) values rounded to bf16 (m = 2n; known spectra). Requests pick a
    matrix uniformly and a window of t in [10, 40] singular values at a uniform position;
    N = 32, L = 32, M = 4. First the capacity: 96 requests submitted at once. Then a Poisson
    stream of `count` requests at min(rate, 0.7 x capacity) per second. Latency is measured
    from submit to result ready (host V_in in, host triplets out)."""
    import threading
    rng = np.random.default_rng(seed)
    mats = []
    for k in range(16):
        rows = int(np.exp(rng.uniform(np.log(1e4), np.log(2e5))))
        c = int(rng.choice([8, 16, 32]))
        nb = max(1, rows // (2 * c))
        mats.append(synth.block_permuted(nb, 2 * c, c, seed=int(rng.integers(1 << 30)), dist="uniform_bf16"))
    spectra = [bp.sigmas_desc() for bp in mats]

    def make(i):
        mi = int(rng.integers(0, 16))
        s = spectra[mi]
        t = int(rng.integers(10, 41))
        first = int(rng.integers(t + 5, s.size - 2 * t - 5))
        a, b, _ = synth.window_interval(s, first, t, min_rel_gap=1e-6, max_shift=10)
        truth = int(((s >= a) & (s <= b)).sum())
        return (mi, a, b, truth, synth.gaussian_block(mats[mi].A.n, 32, 7000 + i))

    srv = B.Server(slots=slots)
    ids = [srv.add_matrix(bp.A) for bp in mats]
    p = B.params(N=32, L=32, M=4)

    def run(reqs, gaps):
        tickets = [None] * len(reqs)
        t0 = time.perf_counter()

        def feeder():
            nxt = t0
            for i, (mi, a, b, truth, V) in enumerate(reqs):
                nxt += gaps[i]
                d = nxt - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                tickets[i] = srv.submit(ids[mi], a, b, p, V)

        th = threading.Thread(target=feeder)
        th.start()
        lat, que, valid = [], [], True
        for i in range(len(reqs)):
            while tickets[i] is None:
                time.sleep(0.0002)
            done, nt, st, l_ms, q_ms = srv.wait(tickets[i])
            stats = srv.take(tickets[i], ids[reqs[i][0]], nt, st).stats
            valid &= (nt == reqs[i][3] and stats["max_res_u"] <= 1e-10 and stats["max_res_v"] <= 1e-10)
            lat.append(l_ms)
            que.append(q_ms)
        t_end = time.perf_counter()
        th.join()
        return len(reqs) / (t_end - t0), lat, que, bool(valid)

    run([make(i) for i in range(16)], np.zeros(16))                      # warm-up
    cap, _, _, valid_cap = run([make(i) for i in range(96)], np.zeros(96))
    lam = min(rate, 0.7 * cap)
    reqs = [make(i) for i in range(count)]
    thr, lat, que, valid = run(reqs, rng.exponential(1.0 / lam, size=count))
    srv.close()
    pct = lambda x, q: float(np.percentile(x, q))
    return {"description": f"16 resident block-permuted matrices (rows 1e4-2e5 log-uniform, 8/16/32 nnz per row, "
                           f"sum rows {sum(bp.A.m for bp in mats)}), windows of t in [10, 40], N=32 L=32 M=4, "
                           f"{slots} slots, HBM budget 80% of free; latency = submit to host result",
            "capacity_solves_per_s": cap, "capacity_all_valid": valid_cap,
            "poisson_rate_per_s": lam, "requests": count, "solves_per_s": thr,
            "latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99), "max": float(np.max(lat))},
            "queue_ms": {"p50": pct(que, 50), "p99": pct(que, 99)}, "all_valid": valid}


def measure_spmm(B, dev, reps=12):
    """The CSR SpMM at full scale, L = 32, on the 2e6 x 1e6 banded-plus-random matrix (32M
    nonzeros, bf16-exact values) and on its known-spectrum twin (62500 permuted 32 x 16 blocks):
    A X and A^T Y in FP64 (FP64 storage), FP32 and double-float (bf16 storage). Three input blocks
    rotate, so no call finds its X in L2 from the call before (as in the Krylov loop, where X is a
    new Lanczos vector every step). Algorithmic bytes per call: (e_a + 4) nnz + 8 (rows + 1) +
    e_x L (m + n), with e_a the stored value size and e_x the block element size (A, X and Y
    once); achieved = bytes / CUDA-event time, against the measured HBM copy bandwidth. The FP64
    product does 2 L flops per nonzero, 1.75 flop/B, against GB300's FP64 balance of ~0.18 flop/B:
    it is bound by the FP64 pipe, and TFLOP/s is reported beside GB/s. The autotuner's pick is
    reported per product."""
    import torch
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm = json.load(open(peaks_path)).get("hbm_gbs", 6780.4) if os.path.exists(peaks_path) else 6780.4
    L = 32
    ctx = B.Context()
    out = {"description": f"L = 32, three rotating inputs; HBM peak {hbm} GB/s (measured copy)"}
    mats = (("banded_random_2000000x1000000", synth.banded_random()),
            ("block_permuted_2000000x1000000", synth.block_permuted(62500, 32, 16, seed=6, dist="uniform_bf16").A))
    for mname, A in mats:
        res = {}
        for storage in ("fp64", "bf16"):
            M = B.Matrix.from_csr(ctx, A, storage=storage)
            Xs = [torch.randn(A.n, L, dtype=torch.float64, device=dev) for _ in range(3)]
            Ys = [torch.randn(A.m, L, dtype=torch.float64, device=dev) for _ in range(3)]
            split = lambda Z: torch.cat([Z.float(), (Z - Z.float().double()).float()], 1).contiguous()
            if storage == "fp64":
                cases = [("A_X_fp64", [lambda X=X: M.spmm(X) for X in Xs], A.m, 8, 8, 0, False),
                         ("At_Y_fp64", [lambda Y=Y: M.spmm(Y, transpose=True) for Y in Ys], A.n, 8, 8, 0, True)]
            else:
                Xf, Yf = [X.float() for X in Xs], [Y.float() for Y in Ys]
                Xd, Yd = [split(X) for X in Xs], [split(Y) for Y in Ys]
                cases = [("A_X_fp32", [lambda X=X: M.spmm_f32(X) for X in Xf], A.m, 2, 4, 1, False),
                         ("At_Y_fp32", [lambda Y=Y: M.spmm_f32(Y, transpose=True) for Y in Yf], A.n, 2, 4, 1, True),
                         ("A_X_df", [lambda X=X: M.spmm_df(X) for X in Xd], A.m, 2, 8, 2, False),
                         ("At_Y_df", [lambda Y=Y: M.spmm_df(Y, transpose=True) for Y in Yd], A.n, 2, 8, 2, True)]
            for cname, fns, rows, e_a, e_x, kind, tr in cases:
                for f in fns:
                    f()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for k in range(reps):
                    fns[k % 3]()
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                byts = (e_a + 4.0) * A.nnz + 8.0 * (rows + 1) + e_x * L * (A.m + A.n)
                res[cname] = {"ms": ms, "algorithmic_bytes": byts, "GB_per_s": byts / ms / 1e6,
                              "frac_of_hbm": byts / ms / 1e6 / hbm, "TFLOP_per_s": 2.0 * A.nnz * L / ms / 1e9,
                              "autotune": B.cmsvd_spmm_tuning(M.handle, tr, kind, L)}
            del Xs, Ys
            M.close()
            torch.cuda.empty_cache()
        res["nnz"] = A.nnz
        out[mname] = res
    ctx.close()
    return out


def measure_table2(B, dev):
    """Exp III (Sec. 4.3, Tables 1-2) on the digit-image stand-in: the eight intervals of
    Table 1 (exterior [a, 1.01] with t = 21, 40, 79, 153; interior windows of t = 17, 39, 85,
    158 values from the 41st), NT variant, N = 32, M = 4, L = 15, 30, 60, 120. Per interval:
    the time of Steps 1-2, 3, 4, 5 and the total, the count, the largest sigma error against
    the dense spectrum and the largest residual."""
    import torch
    A = synth.digits_like()
    s = np.linalg.svd(A.to_dense(), compute_uv=False)
    ctx = B.Context()
    M = B.Matrix.from_csr(ctx, A)
    rows = []
    for kind, t, L in (("exterior", 21, 15), ("exterior", 40, 30), ("exterior", 79, 60), ("exterior", 153, 120),
                       ("interior", 17, 15), ("interior", 39, 30), ("interior", 85, 60), ("interior", 158, 120)):
        if kind == "exterior":
            a, b = 0.5 * (s[t - 1] + s[t]), 1.01 * s[0]
        else:
            a, b, _ = synth.window_interval(s, 40, t)
        truth = np.sort(s[(s >= a) & (s <= b)])
        p = B.params(N=32, L=L, M=4, ell=1, variant="nt", norm_A=float(s[0]))
        Vin = torch.from_numpy(synth.gaussian_block(A.n, L, 5)).to(dev)
        ws = M.workspace(p)
        for rep in range(2):   # the first solve warms up (graph capture)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            status, r = B.cmsvd_solve_interval(M.handle, a, b, p, Vin, ws)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            st = B.cmsvd_result_stats(r)
            k = B.cmsvd_result_count(r)
            sig = np.zeros(k)
            B.cmsvd_result_copy(r, sig)
            B.cmsvd_result_destroy(r)
        err = float(np.max(np.abs(sig - truth) / truth)) if k == truth.size and k else None
        rows.append({"kind": kind, "a": float(a), "b": float(b), "t": int(truth.size), "L": L, "found": int(k),
                     "solver": {1: "krylov", 2: "direct", 3: "dense"}.get(st["solver_used"], "?"),
                     "ms_steps_1_2": st["ms_solve"], "ms_step_3": st["ms_truncate"], "ms_step_4": st["ms_qr"],
                     "ms_step_5": st["ms_ritz"], "ms_total": 1e3 * wall, "lanczos_steps": int(st["krylov_iters"]),
                     "sigma_rel_err": err, "max_res": st["max_res_u"]})
    M.close()
    ctx.close()
    return {"description": "Exp III stand-in: 60000x784 digit-image matrix (synth.digits_like, ~150 nnz/row, "
                           "||A||_2 = 1), Table 1 intervals, NT, N=32 M=4", "rows": rows}


def aggregate_profile(stats):
    """Per kernel class: total event-timed ms and launches over the timed steps."""
    from paper_2109_13655_gb300 import binding as B
    out = {}
    for s in stats:
        for i, name in enumerate(B.PROFILE_CLASSES):
            ms, n = s["prof_ms"][i], s["prof_launches"][i]
            if n:
                d = out.setdefault(name, {"ms": 0.0, "launches": 0, "bytes": 0.0, "flops": 0.0})
                d["ms"] += ms
                d["launches"] += n
                d["bytes"] += s["prof_bytes"][i]
                d["flops"] += s["prof_flops"][i]
    return out


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, mean over the launches
# of one solve of the 200000 x 100000 workload, one ncu capture) for the kernels whose code
# has not changed since; None elsewhere.
MEASURED_TRAFFIC = {
    # k_jacobi_coop, first SVD of a solve (238 columns): 1.92 MB read + 0.58 MB written; the
    # class's algorithmic bytes are its L2 traffic (the columns move through L2 every round)
    ("block_permuted_200000x100000", "jacobi"): 2.50e6,
}


def roofline(dom, prof, stats, w):
    """Roofline of the dominant kernel class: algorithmic bytes or FP64 flops per launch
    (counted by the library for every launch) over its event-timed duration."""
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm = 6780.4
    src = "fallback"
    if os.path.exists(peaks_path):
        hbm = json.load(open(peaks_path)).get("hbm_gbs", hbm)
        src = "measured"
    d = prof[dom]
    sec = d["ms"] / 1e3
    fp64_peak = 152 * 2 * 2 * 2.07e9 / 1e12      # TFLOP/s: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz
    if dom in ("gram", "gemm"):
        # the tall Gram and product run as 36 exact BF16 slice products each (levels p + q <= 9 of
        # 8 slices) on the tensor cores; the class's flops are counted as FP64 products
        bf16 = 1689.0
        bsrc = "fallback"
        if os.path.exists(peaks_path):
            bf16 = json.load(open(peaks_path)).get("bf16_tflops_sustained", bf16)
            bsrc = "measured"
        ach = 36.0 * d["flops"] / sec / 1e12
        return {"kernel": dom, "bound": "tensor", "achieved": ach, "peak": bf16, "unit": "TFLOP/s",
                "frac": ach / bf16, "traffic": MEASURED_TRAFFIC.get((w.get("name"), dom)),
                "fp64_equivalent_tflops": d["flops"] / sec / 1e12,
                "peak_source": f"{bsrc} bf16_tflops_sustained (slice GEMMs inside a long step); achieved counts "
                               "36 BF16 slice products per FP64 product, the slicing and epilogues included",
                "ms_per_launch": d["ms"] / d["launches"]}
    ai = d["flops"] / max(d["bytes"], 1.0)
    if ai > fp64_peak * 1e12 / (hbm * 1e9):
        ach = d["flops"] / sec / 1e12
        return {"kernel": dom, "bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": ach / fp64_peak, "traffic": MEASURED_TRAFFIC.get((w.get("name"), dom)),
                "algorithmic_bytes_per_launch": d["bytes"] / d["launches"],
                "peak_source": "FP64 FMA pipe: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz (derived; probe measured 1.20)",
                "flops_per_launch": d["flops"] / d["launches"], "ms_per_launch": d["ms"] / d["launches"]}
    ach = d["bytes"] / sec / 1e9
    return {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "traffic": None, "peak_source": f"{src} hbm_gbs",
            "bytes_per_launch": d["bytes"] / d["launches"], "ms_per_launch": d["ms"] / d["launches"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="block_permuted_200000x100000")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-krylov", dest="krylov", action="store_false",
                    help="skip the secondary FP64-vs-mixed measurement of the Krylov workload")
    ap.add_argument("--no-batched", dest="batched", action="store_false",
                    help="skip the secondary 64-problem batched measurement")
    ap.add_argument("--no-serving", dest="serving", action="store_false",
                    help="skip the secondary Poisson-arrival serving measurement")
    ap.add_argument("--no-spmm", dest="spmm", action="store_false",
                    help="skip the secondary full-scale SpMM bandwidth measurement")
    ap.add_argument("--no-c3", dest="c3", action="store_false",
                    help="skip the secondary 2e6 x 1e6 mixed-vs-FP64 Krylov measurement (about 3 minutes)")
    ap.add_argument("--table2", action="store_true",
                    help="also run the eight Exp III intervals on the digit-image stand-in (minutes)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    w = workload(args.workload)
    if args.impl == "reference":
        run_reference(args, w, rank)
    else:
        run_ours(args, w, rank, world, local_rank)


if __name__ == "__main__":
    main()
