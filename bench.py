#!/usr/bin/env python
"""Benchmark: H^2 construction from Hessian-vector products + multi-RHS H^2 matvec on GB300.

One step = the whole hot path on the 256 x 256 heat-equation Hessian (N = 65,536,
4,096 sensors, kappa 0.01, T 0.5, sigma 0.01, KD leaves of 64, strong admissibility
0.7, rank cap 32, adaptive peeling to relative tolerance 1e-6), i.e. one FP64
construction followed by FP64 matvecs with nrhs = 1, 32 and 256 resident in HBM.
`value` is the matvec throughput in algorithmic GB/s (stored factor bytes + X and Y
bytes per matvec, summed over the three matvecs, divided by their device time);
the construction time per step is reported as build_s.  The factors (about 0.5 GB)
are larger than L2, so no flush is needed between matvecs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With --impl reference the oracle (CPU, FP64) is timed on a bounded sample of the
same workload (see cpu_baseline) and the same JSON line is printed with
"impl": "reference".  Multi-GPU runs are replicas only (one independent H^2 per rank).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "H² matvec GB/s (% HBM peak) & peeling build s at 1e-6 rel err vs FP64 plain"
CFG = W.MEDIUM_N256
# DRAM bytes (read + write) per gemm_tiles_kernel launch of the bench command, from an ncu capture
# of every launch of that kernel (dram__bytes_read.sum + dram__bytes_write.sum, 1,510 launches);
# reset to None whenever the kernel changes
GEMM_TRAFFIC_PER_LAUNCH = 27.32e6
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
FP64_FLOP_PER_CLK_PER_SM = 4.0   # 2 FP64 FMA per clock per SM (GB300 nominal 1.25 TFLOP/s)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm, src = 6800.0, "fallback"
    try:
        with open(path) as f:
            d = json.load(f)
        hbm, src = float(d["hbm_gbs"]), "measured"
    except Exception:
        pass
    fp64 = SM_COUNT * FP64_FLOP_PER_CLK_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
    return hbm, src, fp64


def matvec_bytes(st: dict, N: int, nrhs: int, elt: int = 8) -> float:
    stored = st["entries_D"] + st["entries_S"] + st["entries_U"] + st["entries_E"]
    return stored * elt + N * nrhs * 2 * elt


def near_flops(st: dict, tree_sizes, nrhs: int) -> float:
    """Flops of the near-field product: every stored off-diagonal near block is applied
    twice (as D and D^T), every diagonal block once."""
    diag = float(np.sum(np.asarray(tree_sizes, dtype=np.float64) ** 2))
    off = st["entries_D"] - diag
    return 2.0 * nrhs * (diag + 2.0 * off)


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu_index: int):
        self.path = os.path.join(tempfile.gettempdir(), f"h2bench_clocks_{os.getpid()}.csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={q}", "--format=csv,noheader",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                mx.append(float(parts[2].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def scaled(cfg: dict, n: int) -> dict:
    """The configuration on an n x n grid with the same sensor fraction (profiling captures)."""
    p = cfg["problem"]
    if n == p.n:
        return cfg
    m = max(1, round(p.m * n * n / p.N))
    return dict(cfg, name=f"{cfg['name']}_at_n{n}", problem=dataclasses.replace(p, n=n, m=m))


def precision_section(h2, torch, stream, bf16_peak: float, n: int = 512) -> dict:
    """512 x 512 heat Hessian (N = 262,144, 16,384 sensors, kappa 0.005, rank cap 48): FP64
    construction, then the matvec with nrhs = 1024 in FP64, TF32 and BF16 (FP32 accumulation,
    near field on tcgen05).  Errors of the reduced-precision results are stated against the
    FP64 matvec of the same H^2.  n other than 512 (profiling) keeps the sensor fraction."""
    c = scaled(W.LARGE_N512, n)
    p, b = c["problem"], c["build"]
    N = p.N
    nrhs = c["nrhs"][0]
    mask = W.sensor_mask(N, p.m, p.sensor_seed)
    gop = h2.HeatOperator(p.n, p.kappa, p.T, p.sigma, mask)
    tree = h2.Tree(W.grid_coords(p.n), b.leaf, b.adm, b.eta)
    opts = h2.default_opts(kmax=b.kmax, q0=b.q0, b_inc=b.b_inc, q_max=b.q_max, adaptive=int(b.adaptive),
                           seed=b.seed, stream=stream, keep_fp32=1, keep_bf16=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    G = h2.H2.build(gop, tree, b.tol, opts)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    st = G.stats()
    gen = torch.Generator(device="cuda").manual_seed(c["rhs_seed"])
    X64 = torch.randn((nrhs, N), dtype=torch.float64, device="cuda", generator=gen)
    Y64 = torch.empty_like(X64)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    G.matvec(X64, Y64, nrhs, h2.H2_FP64, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    out = {"workload": c["name"], "N": N, "nrhs": nrhs, "build_s": build_s, "samples": st["samples"],
           "max_rank": st["max_rank"], "modes": {"FP64": {"ms": e0.elapsed_time(e1)}}}
    _, sizes = tree.boxes(tree.L)
    nflops = near_flops(st, sizes, nrhs)
    for name, mode, xdt, peak in (("TF32", h2.H2_TF32, torch.float32, bf16_peak / 2.0),
                                  ("TF32X3", h2.H2_TF32X3, torch.float32, bf16_peak / 2.0),
                                  ("BF16", h2.H2_BF16, torch.bfloat16, bf16_peak)):
        X = X64.to(xdt)
        Y = torch.empty((nrhs, N), dtype=torch.float32, device="cuda")
        G.matvec(X, Y, nrhs, mode, stream=stream)          # warm-up
        torch.cuda.synchronize()
        G.profile(True)
        reps = 3
        e0.record(stream)
        for _ in range(reps):
            G.matvec(X, Y, nrhs, mode, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = G.profile_read()
        G.profile(False)
        ms = e0.elapsed_time(e1) / reps
        near_ms = prof["near"][0] / max(prof["near"][1], 1)
        err = float((Y.double() - Y64).norm() / Y64.norm())
        # split TF32 runs three products per useful one: the tensor rate counts all three
        tf = nflops * (3 if mode == h2.H2_TF32X3 else 1) / (near_ms / 1e3) / 1e12
        out["modes"][name] = {"ms": ms, "near_ms": near_ms, "near_TFLOPs": tf, "near_frac_of_peak": tf / peak,
                              "peak_TFLOPs": peak, "rel_err_vs_fp64_matvec": err,
                              "stage_ms": {k: v[0] / max(v[1], 1) for k, v in prof.items()}}
        del X, Y
    # FP32 storage at nrhs = 1: the HBM-bound form of the matvec
    x1 = X64[:1].float().contiguous()
    y1 = torch.empty_like(x1)
    G.matvec(x1, y1, 1, h2.H2_FP32, stream=stream)
    reps = 20
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        G.matvec(x1, y1, 1, h2.H2_FP32, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms1 = e0.elapsed_time(e1) / reps
    by1 = matvec_bytes(st, N, 1, 4)
    hbm = peaks()[0]
    out["modes"]["FP32_nrhs1"] = {"ms": ms1, "GBps": by1 / (ms1 / 1e3) / 1e9,
                                  "frac_of_hbm": by1 / (ms1 / 1e3) / 1e9 / hbm, "hbm_peak_GBps": hbm}
    assert G.device_status() == h2.H2_OK
    del X64, Y64
    G.close()
    torch.cuda.empty_cache()
    return out


def batching_section(h2, torch, stream) -> dict:
    """64 heat Hessians of uneven sizes (n ~ U{64..256}, kappa ~ U[0.002, 0.05], 5-20 % sensors):
    batched FP64 construction and the merged, autotuned, graph-captured FP32 matvec with
    nrhs = 64, against the plain FP64 form (one h2_build and one FP64 h2_matvec per Hessian);
    the batched tensor-core forms in TF32 and split TF32 (FP32-grade) beside it."""
    probs = W.batch_problems(64)
    b = CFG["build"]
    nrhs = 64
    ops = [h2.HeatOperator(p.n, p.kappa, p.T, p.sigma, W.sensor_mask(p.N, p.m, p.sensor_seed)) for p in probs]
    trees = [h2.Tree(W.grid_coords(p.n), b.leaf, b.adm, b.eta) for p in probs]
    opts = h2.default_opts(kmax=b.kmax, q0=b.q0, b_inc=b.b_inc, q_max=b.q_max, adaptive=int(b.adaptive),
                           seed=b.seed, keep_fp32=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Gs = h2.build_batched(ops, trees, b.tol, opts)
    torch.cuda.synchronize()
    t_batched = time.perf_counter() - t0
    plain_opts = h2.default_opts(kmax=b.kmax, q0=b.q0, b_inc=b.b_inc, q_max=b.q_max, adaptive=int(b.adaptive),
                                 seed=b.seed, stream=stream)
    t0 = time.perf_counter()
    plain = [h2.H2.build(op, t, b.tol, plain_opts) for op, t in zip(ops, trees)]
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    gen = torch.Generator(device="cuda").manual_seed(77)
    X64 = [torch.randn((nrhs, p.N), dtype=torch.float64, device="cuda", generator=gen) for p in probs]
    X32 = [x.float() for x in X64]
    Y64 = [torch.empty_like(x) for x in X64]
    Y32 = [torch.empty_like(x) for x in X32]
    B = h2.Batch(Gs)
    B.matvec(X32, Y32, nrhs, h2.H2_FP32, stream=stream)     # autotune + capture
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        B.matvec(X32, Y32, nrhs, h2.H2_FP32, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t_bmv = e0.elapsed_time(e1) / reps
    e0.record(stream)
    for _ in range(reps):
        for G, X, Y in zip(plain, X64, Y64):
            G.matvec(X, Y, nrhs, h2.H2_FP64, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t_pmv = e0.elapsed_time(e1) / reps
    err = max(float((y32.double() - y64).norm() / y64.norm()) for y32, y64 in zip(Y32, Y64))
    # TF32 tensor cores: per-handle tcgen05 products between the merged SIMT sweeps
    YT = [torch.empty_like(x) for x in X32]
    B.matvec(X32, YT, nrhs, h2.H2_TF32, stream=stream)     # autotune + capture
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        B.matvec(X32, YT, nrhs, h2.H2_TF32, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t_tc = e0.elapsed_time(e1) / reps
    err_tc = max(float((yt.double() - y64).norm() / y64.norm()) for yt, y64 in zip(YT, Y64))
    # split TF32 on tensor cores: FP32-grade accuracy (the alternative to the FP32 SIMT form)
    Y3 = [torch.empty_like(x) for x in X32]
    B.matvec(X32, Y3, nrhs, h2.H2_TF32X3, stream=stream)     # capture
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        B.matvec(X32, Y3, nrhs, h2.H2_TF32X3, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t_x3 = e0.elapsed_time(e1) / reps
    err_x3 = max(float((y3.double() - y64).norm() / y64.norm()) for y3, y64 in zip(Y3, Y64))
    by32 = sum(matvec_bytes(G.stats(), p.N, nrhs, 4) for G, p in zip(Gs, probs))
    by64 = sum(matvec_bytes(G.stats(), p.N, nrhs, 8) for G, p in zip(plain, probs))
    hbm = peaks()[0]
    out = {"workload": "heat2d_batch64_n64-256", "hessians": len(probs), "N_total": sum(p.N for p in probs),
           "nrhs": nrhs, "build_batched_s": t_batched, "build_plain_fp64_s": t_plain,
           "build_speedup": t_plain / t_batched,
           "matvec_batched_fp32_ms": t_bmv, "matvec_plain_fp64_ms": t_pmv, "matvec_speedup": t_pmv / t_bmv,
           "matvec_batched_GBps": by32 / (t_bmv / 1e3) / 1e9, "matvec_plain_GBps": by64 / (t_pmv / 1e3) / 1e9,
           "rhs_tile_autotuned": B.tuned(nrhs, h2.H2_FP32), "rel_err_fp32_vs_fp64_max": err,
           "matvec_batched_tf32_tc_ms": t_tc, "matvec_batched_tf32_tc_GBps": by32 / (t_tc / 1e3) / 1e9,
           "matvec_batched_tf32_tc_frac_of_hbm": by32 / (t_tc / 1e3) / 1e9 / hbm,
           "matvec_tf32_tc_speedup_vs_plain_fp64": t_pmv / t_tc, "rel_err_tf32_vs_fp64_max": err_tc,
           "matvec_batched_tf32x3_tc_ms": t_x3, "rel_err_tf32x3_vs_fp64_max": err_x3,
           "samples_total": sum(G.stats()["samples"] for G in Gs)}
    B.close()
    for G in Gs + plain:
        G.close()
    torch.cuda.empty_cache()
    return out


def max_over_ranks(x: float, dist) -> float:
    """The largest value of x over the ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(units_per_rank: float, seconds_per_rank: float, dist) -> float:
    """Whole-job throughput of independent replicas: the units of all ranks over the slowest rank's time."""
    world = dist.get_world_size() if dist is not None else 1
    return units_per_rank * world / max_over_ranks(seconds_per_rank, dist)


def rel_err_2norm(h2, torch, gop, G, N: int, norm_est: float, stream) -> float:
    """||H - H~||_2 / ||H||_2 by power iteration through the GPU operator and the FP64 matvec."""
    v = torch.randn(N, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    w1 = torch.empty_like(v)
    w2 = torch.empty_like(v)
    lam, prev = 0.0, 0.0
    v /= v.norm()
    for it in range(60):
        gop.apply(v, w1, 1, stream=stream)
        G.matvec(v, w2, 1, h2.H2_FP64, stream=stream)
        w = w1 - w2
        lam = float(w.norm())
        if lam == 0:
            break
        v = w / lam
        if it > 0 and abs(lam - prev) <= 1e-2 * lam:
            break
        prev = lam
    return lam / norm_est


def learned_ranks_section(h2, torch, stream) -> dict:
    """Rank model trained on adaptive builds of 500 heat Hessians at 128 x 128 (kappa ~ U[0.002,
    0.05], 5-20 % sensors; fine probing q0 16, b_inc 8), then the 256 x 256 and 512 x 512
    Hessians built from the predicted per-level start counts (pad 8, first test 8 columns)
    against plain adaptive peeling (q0 32, b_inc 16), each at tol 1e-6."""
    b = CFG["build"]
    probs = W.batch_problems(500, seed=2025, n_lo=128, n_hi=128)
    fine = h2.default_opts(kmax=b.kmax, q0=16, b_inc=8, q_max=b.q_max, adaptive=1, seed=b.seed)
    feats, targ = [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c0 in range(0, len(probs), 100):          # 100 Hessians per batched call
        chunk = probs[c0:c0 + 100]
        ops = [h2.HeatOperator(q.n, q.kappa, q.T, q.sigma, W.sensor_mask(q.N, q.m, q.sensor_seed)) for q in chunk]
        trees = [h2.Tree(W.grid_coords(q.n), b.leaf, b.adm, b.eta) for q in chunk]
        Gs = h2.build_batched(ops, trees, b.tol, fine)
        for q, t, G in zip(chunk, trees, Gs):
            f = h2.rank_features(t, q.kappa * q.T, q.m / q.N, b.tol)
            lv, tg = h2.rank_targets(G.stats())
            feats.append(f[lv])
            targ += tg
            G.close()
        del ops, trees, Gs
    t_data = time.perf_counter() - t0
    X = torch.from_numpy(np.concatenate(feats).astype(np.float32)).cuda()
    y = torch.from_numpy(np.asarray(targ, dtype=np.float32)).cuda()
    model = h2.RankModel(seed=1, bf16=True)
    p0 = model.get()[0]
    p0[-1] = float(y.mean())
    model.set(p0)
    steps = 4000
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    model.train(X, y, steps, 128, 3e-3, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t_train_ms = e0.elapsed_time(e1)
    loss, _ = model.loss_grad(X, y)
    out = {"train_workload": "heat2d_n128 x 500 (adaptive q0 16, b_inc 8)", "train_rows": int(y.numel()),
           "train_data_build_s": t_data, "train_steps": steps, "train_batch": 128, "train_ms": t_train_ms,
           "train_launches": 1, "train_loss_log2": loss, "eval": {}}
    for cfg in (W.MEDIUM_N256, W.LARGE_N512):
        p, bb = cfg["problem"], cfg["build"]
        gop = h2.HeatOperator(p.n, p.kappa, p.T, p.sigma, W.sensor_mask(p.N, p.m, p.sensor_seed))
        tree = h2.Tree(W.grid_coords(p.n), bb.leaf, bb.adm, bb.eta)
        ql, yl = model.q_levels(tree, p.kappa * p.T, p.m / p.N, bb.tol, pad=8, q_max=bb.q_max)
        base = dict(kmax=bb.kmax, q0=bb.q0, b_inc=bb.b_inc, q_max=bb.q_max, adaptive=1, seed=bb.seed, stream=stream)
        res = {"q_start": [int(v) for v in ql], "predicted_log2": [round(float(v), 3) for v in yl]}
        for key, opts in (("adaptive", h2.default_opts(**base)),
                          ("learned", h2.default_opts(**base, q_level=ql, q_test=8))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            G = h2.H2.build(gop, tree, bb.tol, opts)
            torch.cuda.synchronize()
            bt = time.perf_counter() - t0
            st = G.stats()
            res[key] = {"op_calls": st["op_calls"], "samples": st["samples"], "range_calls": st["range_calls"],
                        "range_probes": st["range_probes"], "range_passed": st["range_passed"], "build_s": bt,
                        "t_peel": st["t_peel"],
                        "rel_err_2norm": rel_err_2norm(h2, torch, gop, G, p.N, st["norm_est"], stream)}
            G.close()
        res["op_calls_saved"] = 1.0 - res["learned"]["op_calls"] / res["adaptive"]["op_calls"]
        res["samples_saved"] = 1.0 - res["learned"]["samples"] / res["adaptive"]["samples"]
        res["build_speedup"] = res["adaptive"]["build_s"] / res["learned"]["build_s"]
        out["eval"][cfg["name"]] = res
        del gop, tree
        torch.cuda.empty_cache()
    model.close()
    return out


def hybrid_section(h2, torch, stream) -> dict:
    """Hybrid construction (Section 3.3, end) on the 256 x 256 and 512 x 512 heat Hessians: a
    global low-rank piece B B^T from an adaptive randomized range finder with several budgets,
    then H^2 on the residual (skipped when the global range test passes), against the plain
    construction, all at tol 1e-6: products, operator calls, build seconds and the 2-norm error
    of each."""
    out = {}
    for cfg, budgets in ((W.MEDIUM_N256, (0, 128, 256, 384, 512)), (W.LARGE_N512, (0, 256, 512, 768))):
        p, bb = cfg["problem"], cfg["build"]
        gop = h2.HeatOperator(p.n, p.kappa, p.T, p.sigma, W.sensor_mask(p.N, p.m, p.sensor_seed))
        tree = h2.Tree(W.grid_coords(p.n), bb.leaf, bb.adm, bb.eta)
        base = dict(kmax=bb.kmax, q0=bb.q0, b_inc=bb.b_inc, q_max=bb.q_max, adaptive=1, seed=bb.seed, stream=stream)
        res = {"runs": {}}
        for budget in budgets:
            opts = h2.default_opts(**base, global_rank=budget)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            G = h2.H2.build(gop, tree, bb.tol, opts)
            torch.cuda.synchronize()
            bt = time.perf_counter() - t0
            st = G.stats()
            key = "plain" if budget == 0 else f"global_{budget}"
            res["runs"][key] = {
                "global_budget": budget, "global_rank": st["range_probes"][0], "global_passed": st["range_passed"][0],
                "samples": st["samples"], "op_calls": st["op_calls"], "build_s": bt, "t_peel": st["t_peel"],
                "t_assemble": st["t_assemble"], "max_rank": st["max_rank"],
                "levels_sampled": sum(1 for l in range(1, st["levels"] + 1) if st["range_passed"][l] != 2),
                "rel_err_2norm": rel_err_2norm(h2, torch, gop, G, p.N, st["norm_est"], stream)}
            G.close()
        plain = res["runs"]["plain"]
        best = min((r for k, r in res["runs"].items() if k != "plain"), key=lambda r: r["samples"])
        res["best"] = {"global_budget": best["global_budget"],
                       "samples_saved": 1.0 - best["samples"] / plain["samples"],
                       "build_speedup": plain["build_s"] / best["build_s"]}
        out[cfg["name"]] = res
        del gop, tree
        torch.cuda.empty_cache()
    return out


def advdiff_section(h2, torch, stream) -> dict:
    """Second Hessian family (Section 4.3's study on a finite-difference stand-in): source
    inversion in stationary advection-diffusion on a 128 x 128 grid, v = (x, y), c = 0.5,
    sigma = 0.01, kappa in {1e-1, 1e-3}, 256 / 1024 / 4096 point observations (nested sets, one
    adjoint solve per observation on the host: the operator's input data), constructed to
    1e-4 in the 2-norm.  Products of the H^2 construction against those of a global low-rank
    approximation (the hybrid's global piece with a budget above n_obs: the adaptive range
    finder and its projection), with build seconds and the 2-norm error of each."""
    from workloads import advdiff as AD
    n, tol, leaf = 128, 1e-4, 64
    N = n * n
    out = {"workload": f"advdiff_n{n}", "tol": tol, "runs": {}}
    tree = h2.Tree(AD.coords(n), leaf, h2.H2_ADM_STRONG, 0.7)
    for kappa in (1e-1, 1e-3):
        t0 = time.perf_counter()
        Zall = AD.hessian_factor(n, kappa, 4096, 11)
        t_solve = time.perf_counter() - t0
        for n_obs in (256, 1024, 4096):
            Zt = torch.from_numpy(np.ascontiguousarray(Zall[:, :n_obs].T)).cuda()
            gop = h2.LowRankOperator(Zt, 1e4)
            row = {"n_obs": n_obs, "kappa": kappa, "adjoint_solves_s": t_solve}
            for key, budget in (("h2", 0), ("global_low_rank", n_obs + 256)):
                opts = h2.default_opts(kmax=48, q0=32, b_inc=16, q_max=512, adaptive=1, seed=7, stream=stream,
                                       global_rank=budget)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                G = h2.H2.build(gop, tree, tol, opts)
                torch.cuda.synchronize()
                bt = time.perf_counter() - t0
                st = G.stats()
                row[key] = {"samples": st["samples"], "op_calls": st["op_calls"], "build_s": bt,
                            "max_rank": max(st["max_rank"]), "global_rank": st["range_probes"][0],
                            "global_passed": st["range_passed"][0],
                            "rel_err_2norm": rel_err_2norm(h2, torch, gop, G, N, st["norm_est"], stream)}
                G.close()
            out["runs"][f"kappa{kappa:g}_obs{n_obs}"] = row
            gop.close()
            del Zt
        del Zall
        torch.cuda.empty_cache()
    return out


def inversion_section(h2, torch, stream) -> dict:
    """Appendix A on the regularised 128 x 128 heat Hessian (N = 16,384, the paper's inversion size):
    A = H~ + beta I with H~ the H^2 approximation (tol 1e-6, leaf 64, strong 0.7) and beta =
    0.01 ||H~|| (condition number about 100); Newton-Schulz with the static threshold, with the
    dynamic threshold (loosest 1e-2), and order-8 hyperpower with the dynamic threshold, each from
    X_0 = I / ||A||_2 to ||A X - I||_2 <= 1e-4 (construction floor 1e-4 / (||A|| ||X_k||), about
    1e-6 near convergence: the paper's construction threshold)."""
    c = scaled(W.MEDIUM_N256, 128)
    p, b = c["problem"], c["build"]
    gop = h2.HeatOperator(p.n, p.kappa, p.T, p.sigma, W.sensor_mask(p.N, p.m, p.sensor_seed))
    tree = h2.Tree(W.grid_coords(p.n), b.leaf, b.adm, b.eta)
    HA = h2.H2.build(gop, tree, b.tol, h2.default_opts(kmax=b.kmax, stream=stream))
    beta = 0.01 * HA.stats()["norm_est"]
    bopts = h2.default_opts(kmax=48, q0=16, b_inc=8, q_max=512, adaptive=1, seed=b.seed, stream=stream)
    eps = 1e-4
    out = {"workload": f"heat2d_n128 regularised, A = H~ + {beta:.4g} I", "N": p.N, "eps": eps, "runs": {}}
    for key, order, loose in (("ns_static", 2, eps), ("ns_dynamic", 2, 1e-2), ("hyperpower8_dynamic", 8, 1e-2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        X, st = h2.invert(HA, shift=beta, order=order, eps=eps, eps_loose=loose, build_opts=bopts)
        torch.cuda.synchronize()
        out["runs"][key] = {"order": order, "eps_loose": loose, "iterations": st["iterations"],
                            "converged": st["converged"], "final_err": st["final_err"],
                            "samples_total": int(sum(st["samples"])), "samples": st["samples"],
                            "seconds": time.perf_counter() - t0, "build_seconds": float(sum(st["t_build"]))}
        X.close()
    out["context_paper_p100_s"] = {"ns_static": 178, "ns_dynamic": 51, "hyperpower8": 20,
                                   "note": "minimal-surface Hessian at n = 16,384 on a P100 (Appendix A); "
                                           "another operator and machine: context only"}
    HA.close()
    torch.cuda.empty_cache()
    return out


def cpu_baseline_sample(n_sample: int = 128, nrhs_list=(1, 32, 256), reps: int = 1) -> dict:
    """The oracle as it stands on a bounded sample of the workload: the same operator family
    (kappa 0.01, 6.25 % sensors, leaf 64, strong 0.7, tol 1e-6) at n = 128, built by the oracle,
    then its matvec timed for nrhs 1, 32, 256 (algorithmic bytes as for the GPU)."""
    import oracle as O

    p = CFG["problem"]
    b = CFG["build"]
    n = n_sample
    m = int(round(p.m * (n * n) / p.N))
    mask = W.sensor_mask(n * n, m, p.sensor_seed)
    op = O.HeatHessian(n, p.kappa, p.T, p.sigma, mask)
    t0 = time.perf_counter()
    h, res = O.build(op, W.grid_coords(n), b.leaf, b.adm, b.eta, b.tol, b.kmax, b.q0, b.b_inc, b.q_max,
                     b.adaptive, b.seed)
    t_build = time.perf_counter() - t0
    ent = O.storage_entries(h)
    st = {"entries_D": ent["D"], "entries_S": ent["S"], "entries_U": ent["U"], "entries_E": ent["E"]}
    tot_bytes, tot_t = 0.0, 0.0
    for nrhs in nrhs_list:
        X = W.rhs(n * n, nrhs, 5)
        for _ in range(reps):
            t0 = time.perf_counter()
            O.matvec(h, X)
            tot_t += time.perf_counter() - t0
            tot_bytes += matvec_bytes(st, n * n, nrhs)
    return {"value": tot_bytes / tot_t / 1e9, "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"oracle build of the same heat-Hessian family at n={n} (N={n * n}, {m} sensors) "
                      f"in {t_build:.1f} s, then oracle matvec with nrhs {list(nrhs_list)} x{reps}",
            "build_s": t_build, "samples": int(res.samples - res.norm_its)}


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O

    p = CFG["problem"]
    b = CFG["build"]
    n = 128
    m = int(round(p.m * (n * n) / p.N))
    mask = W.sensor_mask(n * n, m, p.sensor_seed)
    op = O.HeatHessian(n, p.kappa, p.T, p.sigma, mask)
    h, res = O.build(op, W.grid_coords(n), b.leaf, b.adm, b.eta, b.tol, b.kmax, b.q0, b.b_inc, b.q_max,
                     b.adaptive, b.seed)
    ent = O.storage_entries(h)
    st = {"entries_D": ent["D"], "entries_S": ent["S"], "entries_U": ent["U"], "entries_E": ent["E"]}
    Xs = {nr: W.rhs(n * n, nr, 5) for nr in CFG["nrhs"]}

    def step():
        by, tt = 0.0, 0.0
        for nr, X in Xs.items():
            t0 = time.perf_counter()
            O.matvec(h, X)
            tt += time.perf_counter() - t0
            by += matvec_bytes(st, n * n, nr)
        return by, tt

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    tb, tt = 0.0, 0.0
    for _ in range(args.steps):
        b_, t_ = step()
        tb += b_
        tt += t_
    wall = time.perf_counter() - t0
    val = tb / tt / 1e9
    sample = (f"oracle matvec (nrhs {list(CFG['nrhs'])}) of the oracle-built H^2 of the same heat-Hessian "
              f"family at n={n} (N={n * n}); the n=256 build does not fit a bounded CPU sample")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": CFG["name"], "N": p.N, "nrhs": list(CFG["nrhs"]), "tol": b.tol},
            "cpu_baseline": {"value": val, "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-batching", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-inversion", action="store_true")
    ap.add_argument("--no-hybrid", action="store_true")
    ap.add_argument("--no-advdiff", action="store_true")
    ap.add_argument("--n", type=int, default=None,
                    help="grid size of the stepped Hessian (profiling captures on smaller cases; bench lines use the default)")
    ap.add_argument("--precision-n", type=int, default=512, help="grid size of the precision section")
    args = ap.parse_args()
    global CFG
    if args.n is not None:
        CFG = scaled(CFG, args.n)
    if args.impl == "reference":
        run_reference(args)
        return

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)

    # CPU baseline before any GPU work of this process (spawned pool not needed: single process)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample()

    import paper_2003_10173_gb300 as h2
    from paper_2003_10173_gb300 import build_lib
    build_lib.build()
    h2.lib()

    p, b = CFG["problem"], CFG["build"]
    N = p.N
    mask = W.sensor_mask(N, p.m, p.sensor_seed)
    gop = h2.HeatOperator(p.n, p.kappa, p.T, p.sigma, mask)
    tree = h2.Tree(W.grid_coords(p.n), b.leaf, b.adm, b.eta)
    stream = torch.cuda.current_stream()
    opts = h2.default_opts(kmax=b.kmax, q0=b.q0, b_inc=b.b_inc, q_max=b.q_max, adaptive=int(b.adaptive),
                           seed=b.seed, stream=stream)
    nrhs_list = list(CFG["nrhs"])
    Xd = {nr: torch.from_numpy(np.ascontiguousarray(W.rhs(N, nr, CFG["rhs_seed"] + nr).T)).cuda()
          for nr in nrhs_list}
    Yd = {nr: torch.empty_like(Xd[nr]) for nr in nrhs_list}

    def step(profile=False):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        G = h2.H2.build(gop, tree, b.tol, opts)
        ev1.record(stream)
        mv = {}
        for nr in nrhs_list:
            a = torch.cuda.Event(enable_timing=True)
            c = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            G.matvec(Xd[nr], Yd[nr], nr, h2.H2_FP64, stream=stream)
            c.record(stream)
            mv[nr] = (a, c)
        return G, (ev0, ev1), mv

    for _ in range(args.warmup):
        G, _, _ = step()
        G.close()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    h2.gemm_profile(True)
    launches0 = h2.launch_count()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t_start.record(stream)
    results = []
    for _ in range(args.steps):
        G, bev, mv = step()
        results.append((G, bev, mv))
    t_end.record(stream)
    torch.cuda.synchronize()
    launches = h2.launch_count() - launches0
    gemm_ms, gemm_flops, gemm_n = h2.gemm_profile_read()
    h2.gemm_profile(False)
    clk = clocks.stop()
    total_ms = max_over_ranks(t_start.elapsed_time(t_end), dist)

    st = results[-1][0].stats()
    build_ms = [bev[0].elapsed_time(bev[1]) for _, bev, _ in results]
    mv_ms = {nr: [mv[nr][0].elapsed_time(mv[nr][1]) for _, _, mv in results] for nr in nrhs_list}
    by = {nr: matvec_bytes(st, N, nr) for nr in nrhs_list}
    tot_bytes = sum(by[nr] * len(mv_ms[nr]) for nr in nrhs_list)
    tot_mv_s = sum(sum(mv_ms[nr]) for nr in nrhs_list) / 1e3
    value = aggregate_throughput(tot_bytes, tot_mv_s, dist) / 1e9
    hbm, hbm_src, fp64 = peaks()

    # roofline of the dominant matvec kernel (leaf expansion + near field) at nrhs = 1, FP64
    Gp = results[-1][0]
    Gp.profile(True)
    for _ in range(5):
        Gp.matvec(Xd[1], Yd[1], 1, h2.H2_FP64, stream=stream)
    prof = Gp.profile_read()
    Gp.profile(False)
    _, sizes = tree.boxes(tree.L)
    nr_ms, nr_n = prof["near"]
    nr_s = nr_ms / nr_n / 1e3
    achieved = near_flops(st, sizes, 1) / nr_s / 1e12
    roofline_matvec = {"bound": "alu", "achieved": achieved, "peak": fp64, "unit": "TFLOP/s",
                       "frac": achieved / fp64, "traffic": None,
                       "kernel": "mv_scatter_kernel<double,...,1,true> (near field, nrhs=1)",
                       "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x 2070 MHz",
                       "hbm_GBps": st["entries_D"] * 8 / nr_s / 1e9}
    # dominant kernel of a step (about two thirds of the device time): the construction's FP64
    # batched GEMM, timed per launch with events on the build stream over the timed steps
    gemm_tf = gemm_flops / (gemm_ms / 1e3) / 1e12 if gemm_ms > 0 else None
    roofline = {"bound": "alu", "achieved": gemm_tf, "peak": fp64, "unit": "TFLOP/s",
                "frac": (gemm_tf / fp64) if gemm_tf else None, "traffic": GEMM_TRAFFIC_PER_LAUNCH,
                "kernel": "gemm_tiles_kernel (FP64 batched GEMM: operator DSTs, piece subtraction, Gram)",
                "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x 2070 MHz",
                "launches": gemm_n, "ms": gemm_ms,
                "flops_per_launch": gemm_flops / max(gemm_n, 1), "ms_per_launch": gemm_ms / max(gemm_n, 1)}
    near_bytes = st["entries_D"] * 8
    hbm_view = {"nrhs1_matvec_GBps": by[1] / (np.mean(mv_ms[1]) / 1e3) / 1e9,
                "frac_of_hbm": by[1] / (np.mean(mv_ms[1]) / 1e3) / 1e9 / hbm, "hbm_peak_GBps": hbm,
                "hbm_peak_source": hbm_src}

    precision = None
    if rank == 0 and not args.no_precision:
        bf16_peak = 1937.9
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                bf16_peak = float(json.load(f)["bf16_tflops"])
        except Exception:
            pass
        precision = precision_section(h2, torch, stream, bf16_peak, args.precision_n)

    batching = None
    if rank == 0 and not args.no_batching:
        batching = batching_section(h2, torch, stream)

    # end to end through the public call with host buffers (pinned) and copies in the timed region
    Gp2 = results[-1][0]
    Xh = {nr: torch.empty((nr, N), dtype=torch.float64, pin_memory=True) for nr in nrhs_list}
    Yh = {nr: torch.empty((nr, N), dtype=torch.float64, pin_memory=True) for nr in nrhs_list}
    for nr in nrhs_list:
        Xh[nr].copy_(Xd[nr].cpu())
    Xe = {nr: torch.empty_like(Xd[nr]) for nr in nrhs_list}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = 3
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        for nr in nrhs_list:
            Xe[nr].copy_(Xh[nr], non_blocking=True)
            Gp2.matvec(Xe[nr], Yd[nr], nr, h2.H2_FP64, stream=stream)
            Yh[nr].copy_(Yd[nr], non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_s = e0.elapsed_time(e1) / 1e3
    e2e_bytes = reps * sum(by[nr] for nr in nrhs_list)
    e2e = {"value": aggregate_throughput(e2e_bytes, e2e_s, dist) / 1e9, "unit": "GB/s",
           "h2d_bytes_per_step": sum(N * nr * 8 for nr in nrhs_list),
           "d2h_bytes_per_step": sum(N * nr * 8 for nr in nrhs_list)}

    # accuracy of the last build (2-norm, power iteration through the GPU matvec and operator)
    rel_err = None
    if rank == 0:
        rel_err = rel_err_2norm(h2, torch, gop, Gp2, N, st["norm_est"], stream)

    learned = None
    if rank == 0 and not args.no_learned:
        learned = learned_ranks_section(h2, torch, stream)

    hybrid = None
    if rank == 0 and not args.no_hybrid:
        hybrid = hybrid_section(h2, torch, stream)

    advdiff = None
    if rank == 0 and not args.no_advdiff:
        advdiff = advdiff_section(h2, torch, stream)

    inversion = None
    if rank == 0 and not args.no_inversion:
        inversion = inversion_section(h2, torch, stream)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": CFG["name"], "N": N, "grid": f"{p.n}x{p.n}", "sensors": p.m, "kappa": p.kappa,
                       "leaf": b.leaf, "adm": "strong", "eta": b.eta, "kmax": b.kmax, "tol": b.tol,
                       "nrhs": nrhs_list, "mode": "FP64",
                       "l2": "H2 factors larger than L2 (no flush needed)", "parallelism": "replicas"},
            "build_s": float(np.mean(build_ms)) / 1e3,
            "rel_err_2norm": rel_err,
            "samples": st["samples"], "norm_products": st["norm_products"], "max_rank": st["max_rank"],
            "range_probes": st["range_probes"], "proj_probes": st["proj_probes"],
            "matvec_ms": {str(nr): float(np.mean(mv_ms[nr])) for nr in nrhs_list},
            "matvec_GBps": {str(nr): by[nr] / (np.mean(mv_ms[nr]) / 1e3) / 1e9 for nr in nrhs_list},
            "stored_bytes_fp64": (st["entries_D"] + st["entries_S"] + st["entries_U"] + st["entries_E"]) * 8,
            "hbm_view": hbm_view,
            "roofline": roofline, "roofline_matvec": roofline_matvec,
            "stage_ms_nrhs1": {k: v[0] / max(v[1], 1) for k, v in prof.items()},
            "build_phase_s": {k: st[k] for k in ("t_norm", "t_op", "t_peel", "t_assemble")},
            "e2e": e2e, "gpu_launches": launches, "clocks": clk,
        }
        if precision is not None:
            line["precision"] = precision
        if batching is not None:
            line["batching"] = batching
        if learned is not None:
            line["learned_ranks"] = learned
        if hybrid is not None:
            line["hybrid"] = hybrid
        if advdiff is not None:
            line["advdiff"] = advdiff
        if inversion is not None:
            line["inversion"] = inversion
        if cpu is not None:
            line["cpu_baseline"] = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")}
        print(json.dumps(line), flush=True)
    for G, _, _ in results:
        G.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
