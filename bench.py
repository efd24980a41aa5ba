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
# The stepped construction keeps each level's range basis to the columns its passing a-posteriori
# test certified (the adaptive range finder's textbook form); the certified_bases section sets
# it against bases that span every probe drawn.  The oracle legs build the same way.
HEADLINE_CERTIFIED = True
# DRAM bytes (read + write) of one mv_leaf_near_kernel launch at nrhs = 256, from an ncu capture of
# the same kernel on the 128 x 128 member of the bench family (profiles/ names the command), with
# the algorithmic bytes of that launch; the full-size traffic is scaled by the algorithmic bytes
# (near-block entries and right-hand-side rows both grow with N).  Recapture after changing the kernel.
MATVEC_TRAFFIC_SMALL = {"dram_bytes": 692778240 + 38321664, "algorithmic_bytes": 1.610e8, "grid": "128x128"}
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
FP64_FLOP_PER_CLK_PER_SM = 4.0   # 2 FP64 FMA per clock per SM (GB300 nominal 1.25 TFLOP/s)


def fp64_peak_measured(torch, stream) -> float:
    """Dense FP64 rate of this GPU: cuBLAS DGEMM (torch.matmul, 4096 x 4096 float64), best of 5,
    CUDA events on the current stream."""
    n = 4096
    g = torch.Generator(device="cuda").manual_seed(1)
    a = torch.randn(n, n, dtype=torch.float64, device="cuda", generator=g)
    b = torch.randn(n, n, dtype=torch.float64, device="cuda", generator=g)
    for _ in range(2):
        torch.matmul(a, b)
    best = float("inf")
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        torch.matmul(a, b)
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    del a, b
    return 2.0 * n ** 3 / best / 1e12


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
    construction, then the matvec with nrhs = 1024 in FP64, TF32, split TF32 and BF16 (FP32
    accumulation, near field on tcgen05) and compensated FP32 (FP32 storage, float-pair
    arithmetic).  Errors of the reduced-precision results are stated against the FP64 matvec of
    the same H^2.  n other than 512 (profiling) keeps the sensor fraction."""
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
    # compensated FP32 (FP32 storage, float-pair arithmetic on the FP32 pipe, FP64 X and Y)
    Yc = torch.empty_like(X64)
    G.matvec(X64, Yc, nrhs, h2.H2_FP32C, stream=stream)          # warm-up
    torch.cuda.synchronize()
    G.profile(True)
    reps = 3
    e0.record(stream)
    for _ in range(reps):
        G.matvec(X64, Yc, nrhs, h2.H2_FP32C, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = G.profile_read()
    G.profile(False)
    msc = e0.elapsed_time(e1) / reps
    errc = float((Yc - Y64).norm() / Y64.norm())
    colc = float(((Yc - Y64).norm(dim=1) / Y64.norm(dim=1)).max())
    out["modes"]["FP32C"] = {"ms": msc, "rel_err_vs_fp64_matvec": errc, "worst_column_rel_err": colc,
                             "speedup_vs_fp64": out["modes"]["FP64"]["ms"] / msc,
                             "stage_ms": {k: v[0] / max(v[1], 1) for k, v in prof.items()}}
    del Yc
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
    the batched tensor-core forms in TF32 and split TF32 (FP32-grade) beside it.  Both
    constructions use the stepped construction's range bases (certified or not)."""
    probs = W.batch_problems(64)
    b = CFG["build"]
    nrhs = 64
    ops = [h2.HeatOperator(p.n, p.kappa, p.T, p.sigma, W.sensor_mask(p.N, p.m, p.sensor_seed)) for p in probs]
    trees = [h2.Tree(W.grid_coords(p.n), b.leaf, b.adm, b.eta) for p in probs]
    opts = h2.default_opts(kmax=b.kmax, q0=b.q0, b_inc=b.b_inc, q_max=b.q_max, adaptive=int(b.adaptive),
                           seed=b.seed, keep_fp32=1, certified=int(HEADLINE_CERTIFIED))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Gs = h2.build_batched(ops, trees, b.tol, opts)
    torch.cuda.synchronize()
    t_batched = time.perf_counter() - t0
    plain_opts = h2.default_opts(kmax=b.kmax, q0=b.q0, b_inc=b.b_inc, q_max=b.q_max, adaptive=int(b.adaptive),
                                 seed=b.seed, stream=stream, certified=int(HEADLINE_CERTIFIED))
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
           "range_bases": "certified" if HEADLINE_CERTIFIED else "all probes",
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
    0.05], 5-20 % sensors; fine probing q0 16, b_inc 8), then the 256 x 256 and 512 x 512 bench
    Hessians and held-out sets (32 Hessians at 256 x 256, 8 at 512 x 512, parameters and sensor
    sets drawn afresh) built from the predicted per-level start counts (pad 8, first test 8
    columns) against plain adaptive peeling (q0 32, b_inc 16), each at tol 1e-6."""
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
            lv, tg = h2.rank_targets(G)
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
    # held-out Hessians of the family (kappa, sensor fraction and sensor sets never trained on):
    # 32 at 256 x 256 and 8 at 512 x 512, each built plain and from the predicted starts
    out["held_out"] = {}
    for n, count, seed, cfg in ((256, 32, 7001, W.MEDIUM_N256), (512, 8, 7002, W.LARGE_N512)):
        bb = cfg["build"]
        base = dict(kmax=bb.kmax, q0=bb.q0, b_inc=bb.b_inc, q_max=bb.q_max, adaptive=1, seed=bb.seed, stream=stream)
        rows = []
        for i, q in enumerate(W.batch_problems(count, seed=seed, n_lo=n, n_hi=n)):
            q = dataclasses.replace(q, sensor_seed=90000 + 100 * n + i)
            gop = h2.HeatOperator(q.n, q.kappa, q.T, q.sigma, W.sensor_mask(q.N, q.m, q.sensor_seed))
            tree = h2.Tree(W.grid_coords(q.n), bb.leaf, bb.adm, bb.eta)
            ql, _ = model.q_levels(tree, q.kappa * q.T, q.m / q.N, bb.tol, pad=8, q_max=bb.q_max)
            row = {"kappa": q.kappa, "sensor_fraction": q.m / q.N}
            for key, opts in (("adaptive", h2.default_opts(**base)),
                              ("learned", h2.default_opts(**base, q_level=ql, q_test=8))):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                G = h2.H2.build(gop, tree, bb.tol, opts)
                torch.cuda.synchronize()
                bt = time.perf_counter() - t0
                st = G.stats()
                row[key] = {"op_calls": st["op_calls"], "samples": st["samples"], "build_s": bt,
                            "rel_err_2norm": rel_err_2norm(h2, torch, gop, G, q.N, st["norm_est"], stream)}
                G.close()
            rows.append(row)
            del gop, tree
        def saved(k):
            return [1.0 - r["learned"][k] / r["adaptive"][k] for r in rows]
        sp = [r["adaptive"]["build_s"] / r["learned"]["build_s"] for r in rows]
        out["held_out"][f"heat{n}"] = {
            "hessians": count, "seed": seed,
            "op_calls_saved_mean": float(np.mean(saved("op_calls"))), "op_calls_saved_min": float(np.min(saved("op_calls"))),
            "samples_saved_mean": float(np.mean(saved("samples"))), "samples_saved_min": float(np.min(saved("samples"))),
            "build_speedup_mean": float(np.mean(sp)), "build_speedup_min": float(np.min(sp)),
            "rel_err_max_adaptive": float(max(r["adaptive"]["rel_err_2norm"] for r in rows)),
            "rel_err_max_learned": float(max(r["learned"]["rel_err_2norm"] for r in rows)),
            "within_1e-6_learned": int(sum(r["learned"]["rel_err_2norm"] <= 1e-6 for r in rows)),
            "within_1e-6_adaptive": int(sum(r["adaptive"]["rel_err_2norm"] <= 1e-6 for r in rows)),
            "per_hessian": rows}
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


def certified_section(h2, torch, stream) -> dict:
    """Certified range bases (the passing range test's columns left out of each level's basis,
    the adaptive range finder's textbook form) against the default bases on the 256 x 256 and
    512 x 512 heat Hessians at tol 1e-6: products, operator calls, build seconds (best of two),
    projection probes, ranks and the 2-norm error of each."""
    out = {}
    for cfg in (W.MEDIUM_N256, W.LARGE_N512):
        p, bb = cfg["problem"], cfg["build"]
        gop = h2.HeatOperator(p.n, p.kappa, p.T, p.sigma, W.sensor_mask(p.N, p.m, p.sensor_seed))
        tree = h2.Tree(W.grid_coords(p.n), bb.leaf, bb.adm, bb.eta)
        res = {}
        for key, c in (("default", 0), ("certified", 1)):
            opts = h2.default_opts(kmax=bb.kmax, q0=bb.q0, b_inc=bb.b_inc, q_max=bb.q_max, adaptive=1, seed=bb.seed,
                                   stream=stream, certified=c)
            best = None
            for _ in range(2):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                G = h2.H2.build(gop, tree, bb.tol, opts)
                torch.cuda.synchronize()
                bt = time.perf_counter() - t0
                if best is None or bt < best[0]:
                    if best is not None:
                        best[1].close()
                    best = (bt, G)
                else:
                    G.close()
            bt, G = best
            st = G.stats()
            res[key] = {"samples": st["samples"], "op_calls": st["op_calls"], "build_s": bt, "t_peel": st["t_peel"],
                        "t_assemble": st["t_assemble"], "proj_probes": st["proj_probes"],
                        "range_probes": st["range_probes"], "max_rank": st["max_rank"], "tol_met": st["tol_met"],
                        "rel_err_2norm": rel_err_2norm(h2, torch, gop, G, p.N, st["norm_est"], stream)}
            G.close()
        res["samples_saved"] = 1.0 - res["certified"]["samples"] / res["default"]["samples"]
        res["build_speedup"] = res["default"]["build_s"] / res["certified"]["build_s"]
        out[cfg["name"]] = res
        del gop, tree
        torch.cuda.empty_cache()
    return out


def update_section(h2, torch, stream, G, N: int, build_s: float) -> dict:
    """Low-rank update with recompression (Section 3.2, Eqs. 3.3-3.4) of the headline H^2 matrix:
    A~ = A + B B^T with a Gaussian B (columns of the size of the Hessian's leading eigenvalues),
    recompressed at tol 1e-6 without any sampling.  Reports the update's seconds (norm estimate
    and recompression), the new ranks, and ||A~_H2 - (A + B B^T)||_2 / ||A + B B^T||_2 by power
    iteration through the two handles' FP64 matvecs, against the construction's own seconds."""
    st0 = G.stats()
    out = {"workload": "heat 256x256 H^2 (the headline build) + B B^T, B Gaussian N x r scaled by "
                       "sqrt(||H||/N)", "tol": 1e-6, "build_s_for_comparison": build_s, "runs": {}}
    gen = torch.Generator("cuda").manual_seed(17)
    for r in (8, 16):
        B = torch.randn((r, N), dtype=torch.float64, device="cuda", generator=gen) * (st0["norm_est"] / N) ** 0.5
        opts = h2.default_opts(kmax=48, stream=stream)
        times = []
        for rep in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Gu = G.lowrank_update(B, r, 1e-6, opts=opts)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
            if rep < 2:
                Gu.close()
        st = Gu.stats()
        v = torch.randn(N, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
        v /= v.norm()
        w1, w2 = torch.empty_like(v), torch.empty_like(v)
        lam, prev = 0.0, 0.0
        for it in range(60):
            G.matvec(v, w1, 1, h2.H2_FP64, stream=stream)
            Gu.matvec(v, w2, 1, h2.H2_FP64, stream=stream)
            torch.cuda.synchronize()
            w = w1 + B.T @ (B @ v) - w2
            lam = float(w.norm())
            if lam == 0:
                break
            v = w / lam
            if it > 0 and abs(lam - prev) <= 1e-2 * lam:
                break
            prev = lam
        out["runs"][f"r{r}"] = {"update_s": float(np.median(times)), "t_norm": st["t_norm"],
                                "t_recompress": st["t_assemble"], "max_rank_before": st0["max_rank"],
                                "max_rank_after": st["max_rank"], "norm_est": st["norm_est"],
                                "rel_err_2norm": lam / st["norm_est"], "tol_met": st["tol_met"]}
        Gu.close()
    return out


def small_section(h2, torch, stream) -> dict:
    """The 32 x 32 configuration (N = 1,024, 200 sensors, leaf 32, 64 fixed probes per level, rank
    cap 16, nrhs 16 in FP64), with the weak (HSS) partition it names and the strong one beside it:
    build seconds, products, ranks, 2-norm error, matvec time and algorithmic GB/s (median of 20)."""
    c = W.SMALL_N32
    p, b = c["problem"], c["build"]
    nrhs = c["nrhs"][0]
    gop = h2.HeatOperator(p.n, p.kappa, p.T, p.sigma, W.sensor_mask(p.N, p.m, p.sensor_seed))
    out = {"workload": c["name"], "N": p.N, "nrhs": nrhs, "runs": {}}
    gen = torch.Generator(device="cuda").manual_seed(c["rhs_seed"])
    X = torch.randn((nrhs, p.N), dtype=torch.float64, device="cuda", generator=gen)
    Y = torch.empty_like(X)
    for name, adm in (("weak", h2.H2_ADM_WEAK), ("strong", h2.H2_ADM_STRONG)):
        tree = h2.Tree(W.grid_coords(p.n), b.leaf, adm, b.eta)
        opts = h2.default_opts(kmax=b.kmax, q0=b.q0, b_inc=b.b_inc, q_max=b.q_max, adaptive=int(b.adaptive),
                               seed=b.seed, stream=stream)
        times = []
        for _ in range(5):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            G = h2.H2.build(gop, tree, b.tol, opts)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
            G.close()
        G = h2.H2.build(gop, tree, b.tol, opts)
        st = G.stats()
        ms = []
        for _ in range(20):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            G.matvec(X, Y, nrhs, h2.H2_FP64, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        mv = float(np.median(ms))
        out["runs"][name] = {"build_s": float(np.median(times)), "samples": st["samples"], "max_rank": st["max_rank"],
                             "tol_met": st["tol_met"], "matvec_ms": mv,
                             "matvec_GBps": matvec_bytes(st, p.N, nrhs) / (mv / 1e3) / 1e9,
                             "rel_err_2norm": rel_err_2norm(h2, torch, gop, G, p.N, st["norm_est"], stream)}
        G.close()
    return out


def sampling_section(h2, torch, stream) -> dict:
    """Sampling structure (Section 3.3: C_l probe blocks of k columns per level).  The weak structure
    (sibling blocks, C_l = 2: range and projection pass, adaptive k) against strong-structure
    coloured sampling (the destination far blocks, C_l = colours + projection slots, k = q0 = 16
    fixed), on the heat Hessians at 64^2 and 128^2 (tol 1e-6, leaf 64, strong eta 0.7): products,
    operator calls, build seconds and the 2-norm error of each; at 256^2 only the coloured plan's
    counts (its products would exceed N)."""
    out = {"q": 16, "runs": {}}
    for n in (64, 128):
        p = W.SMALL_N32["problem"]
        gop = h2.HeatOperator(n, p.kappa, p.T, p.sigma, W.sensor_mask(n * n, p.m, p.sensor_seed))
        tree = h2.Tree(W.grid_coords(n), 64, h2.H2_ADM_STRONG, 0.7)
        res = {"plan": tree.colored_plan(16)}
        for name, kw in (("weak", dict(q0=32, b_inc=16, q_max=256)),
                         ("colored", dict(q0=16, sampling=h2.H2_SAMPLING_COLORED))):
            opts = h2.default_opts(kmax=32, seed=7, stream=stream, **kw)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            G = h2.H2.build(gop, tree, 1e-6, opts)
            torch.cuda.synchronize()
            st = G.stats()
            res[name] = {"samples": st["samples"], "op_calls": st["op_calls"], "build_s": time.perf_counter() - t0,
                         "t_op": st["t_op"], "range_probes": st["range_probes"][:st["levels"] + 1],
                         "proj_probes": st["proj_probes"][:st["levels"] + 1], "max_rank": st["max_rank"][:st["levels"] + 1],
                         "rel_err_2norm": rel_err_2norm(h2, torch, gop, G, n * n, st["norm_est"], stream)}
            G.close()
        res["products_ratio_colored_over_weak"] = res["colored"]["samples"] / res["weak"]["samples"]
        out["runs"][f"heat{n}"] = res
        del gop, tree
        torch.cuda.empty_cache()
    t256 = h2.Tree(W.grid_coords(256), 64, h2.H2_ADM_STRONG, 0.7)
    pl = t256.colored_plan(16)
    out["plan_256"] = dict(pl, products=16 * (sum(pl["colors"]) + sum(pl["slots"])) + 64 * pl["leaf_colors"])
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
    1e-6 near convergence: the paper's construction threshold).  Then the warm-started inversion of
    a nearby Hessian from that inverse: Newton-Schulz iterations against unrolled ones."""
    c = scaled(W.MEDIUM_N256, 128)
    p, b = c["problem"], c["build"]
    gop = h2.HeatOperator(p.n, p.kappa, p.T, p.sigma, W.sensor_mask(p.N, p.m, p.sensor_seed))
    tree = h2.Tree(W.grid_coords(p.n), b.leaf, b.adm, b.eta)
    HA = h2.H2.build(gop, tree, b.tol, h2.default_opts(kmax=b.kmax, stream=stream))
    beta = 0.01 * HA.stats()["norm_est"]
    bopts = h2.default_opts(kmax=48, q0=16, b_inc=8, q_max=512, adaptive=1, seed=b.seed, stream=stream)
    eps = 1e-4
    out = {"workload": f"heat2d_n128 regularised, A = H~ + {beta:.4g} I", "N": p.N, "eps": eps, "runs": {}}
    def record(key, st, t0, **extra):
        out["runs"][key] = {"iterations": st["iterations"], "converged": st["converged"],
                            "final_err": st["final_err"], "samples_total": int(sum(st["samples"])),
                            "samples": st["samples"], "seconds": time.perf_counter() - t0,
                            "build_seconds": float(sum(st["t_build"])), **extra}

    prev = None
    for key, order, loose in (("ns_static", 2, eps), ("ns_dynamic", 2, 1e-2), ("hyperpower8_dynamic", 8, 1e-2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        X, st = h2.invert(HA, shift=beta, order=order, eps=eps, eps_loose=loose, build_opts=bopts)
        torch.cuda.synchronize()
        record(key, st, t0, order=order, eps_loose=loose)
        if key == "ns_dynamic":
            prev = X
        else:
            X.close()
    # Warm start (Appendix A: the next optimisation iterate's Hessian, inverted from the previous
    # inverse): the same family with kappa 5 % larger; Newton-Schulz from X_0 = the previous inverse
    # against the unrolled iterations (k steps in one construction)
    gop2 = h2.HeatOperator(p.n, 1.05 * p.kappa, p.T, p.sigma, W.sensor_mask(p.N, p.m, p.sensor_seed))
    HB = h2.H2.build(gop2, tree, b.tol, h2.default_opts(kmax=b.kmax, stream=stream))
    out["warm_start"] = {"workload": "A' = H~' + beta I, H~' of the same family with kappa x 1.05; X_0 = the "
                                     "ns_dynamic inverse of A"}
    for key, kw in (("warm_ns_static", dict(order=2, eps_loose=eps)), ("warm_ns_dynamic", dict(order=2, eps_loose=1e-2)),
                    ("warm_unrolled_2", dict(unroll=2, eps_loose=eps)), ("warm_unrolled_3", dict(unroll=3, eps_loose=eps))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        X, st = h2.invert(HB, shift=beta, eps=eps, build_opts=bopts, x0=prev, **kw)
        torch.cuda.synchronize()
        record(key, st, t0, start_err=st["err"][0], **kw)
        X.close()
    prev.close()
    HB.close()
    out["context_paper_p100_s"] = {"ns_static": 178, "ns_dynamic": 51, "hyperpower8": 20,
                                   "note": "minimal-surface Hessian at n = 16,384 on a P100 (Appendix A); "
                                           "another operator and machine: context only"}
    HA.close()
    torch.cuda.empty_cache()
    return out


def _spec(cfg: dict, nrhs) -> dict:
    p, b = cfg["problem"], cfg["build"]
    return {"n": p.n, "m": p.m, "kappa": p.kappa, "T": p.T, "sigma": p.sigma, "sensor_seed": p.sensor_seed,
            "leaf": b.leaf, "adm": b.adm, "eta": b.eta, "tol": b.tol, "kmax": b.kmax, "q0": b.q0, "b_inc": b.b_inc,
            "q_max": b.q_max, "adaptive": bool(b.adaptive), "seed": b.seed, "nrhs": list(nrhs), "rhs_seed": 5,
            "certified": HEADLINE_CERTIFIED}


def oracle_worker(spec: dict) -> dict:
    """The oracle as it stands, in this process: build the configuration's H^2 (or load its factors
    from spec["load"]), then time its matvec for every nrhs (reps times).  Returns times, bytes and
    counts; spec["dump"] saves the factors for a later worker."""
    import oracle as O

    n = spec["n"]
    N = n * n
    out = {"threads_env": os.environ.get("OMP_NUM_THREADS"), "cores": os.cpu_count()}
    if spec.get("load"):
        z = np.load(spec["load"])
        tree = O.ClusterTree(W.grid_coords(n), spec["leaf"])
        h = O.from_factor_arrays(tree, O.Partition(tree, spec["adm"], spec["eta"]), z["ranks"], z["U"], z["E"], z["S"],
                                 z["D"])
        out["build_s"] = None
    else:
        mask = W.sensor_mask(N, spec["m"], spec["sensor_seed"])
        op = O.HeatHessian(n, spec["kappa"], spec["T"], spec["sigma"], mask)
        t0 = time.perf_counter()
        h, res = O.build(op, W.grid_coords(n), spec["leaf"], spec["adm"], spec["eta"], spec["tol"], spec["kmax"],
                         spec["q0"], spec["b_inc"], spec["q_max"], spec["adaptive"], spec["seed"],
                         certified=bool(spec.get("certified", False)))
        out["build_s"] = time.perf_counter() - t0
        out["samples"] = int(res.samples - res.norm_its)
        if spec.get("dump"):
            r, U, E, S, D = O.factor_arrays(h)
            np.savez(spec["dump"], ranks=r, U=U, E=E, S=S, D=D)
    ent = O.storage_entries(h)
    st = {"entries_D": ent["D"], "entries_S": ent["S"], "entries_U": ent["U"], "entries_E": ent["E"]}
    out["matvec_s"], out["bytes"] = {}, {}
    for nr in spec["nrhs"]:
        X = W.rhs(N, nr, spec["rhs_seed"])
        ts = []
        for _ in range(spec.get("reps", 1)):
            t0 = time.perf_counter()
            O.matvec(h, X)
            ts.append(time.perf_counter() - t0)
        out["matvec_s"][str(nr)] = ts
        out["bytes"][str(nr)] = matvec_bytes(st, N, nr)
    return out


def run_oracle_worker(spec: dict, threads: int | None = None, timeout: float = 1800.0) -> dict:
    """oracle_worker in a child process (so that the BLAS thread count can be fixed at start-up)."""
    env = dict(os.environ)
    if threads is not None:
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[k] = str(threads)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-worker", json.dumps(spec)], env=env,
                       capture_output=True, text=True, timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError(f"oracle worker failed: {r.stderr[-2000:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


def gbps(res: dict) -> float:
    by = sum(res["bytes"][k] * len(v) for k, v in res["matvec_s"].items())
    return by / sum(sum(v) for v in res["matvec_s"].values()) / 1e9


def oracle_side_measurements(main_res: dict | None = None, dump: str | None = None) -> dict:
    """The oracle beyond the headline sample: its matvec at one thread on the factors it built
    (loaded from `dump`), and the 32 x 32 configuration (weak partition, 64 fixed probes,
    nrhs 16) built and applied at all cores and at one thread."""
    out = {}
    if dump:
        one = run_oracle_worker(dict(_spec(CFG, CFG["nrhs"]), load=dump), threads=1)
        out["headline_matvec_1thread_GBps"] = gbps(one)
        out["headline_matvec_1thread_s"] = {k: float(np.mean(v)) for k, v in one["matvec_s"].items()}
    for th, key in ((None, "nproc"), (1, "1thread")):
        r = run_oracle_worker(dict(_spec(W.SMALL_N32, W.SMALL_N32["nrhs"]), reps=3), threads=th)
        out[f"small_n32_{key}"] = {"build_s": r["build_s"], "matvec_GBps": gbps(r), "samples": r["samples"],
                                   "threads": th or os.cpu_count()}
    return out


def cpu_baseline_full() -> dict:
    """The oracle as it stands on the headline workload itself: the FP64 construction of the
    256 x 256 Hessian (once; its time is reported as build_s), then its matvec with nrhs 1, 32,
    256 (the sample the value is measured on), at all host cores; plus one-thread and 32 x 32
    measurements (oracle_side_measurements)."""
    dump = os.path.join(tempfile.gettempdir(), f"h2bench_oracle_{os.getpid()}.npz")
    try:
        res = run_oracle_worker(dict(_spec(CFG, CFG["nrhs"]), dump=dump))
        side = oracle_side_measurements(res, dump)
    finally:
        if os.path.exists(dump):
            os.remove(dump)
    mv = {k: float(np.mean(v)) for k, v in res["matvec_s"].items()}
    return {"value": gbps(res), "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"oracle matvec with nrhs {list(CFG['nrhs'])} of the oracle-built H^2 of the headline workload "
                      f"({CFG['name']}, N={CFG['problem'].N}); the oracle construction itself took "
                      f"{res['build_s']:.1f} s at {os.cpu_count()} cores",
            "same_config": True, "build_s": res["build_s"], "samples": res["samples"], "matvec_s": mv, **side}


def run_reference(args) -> None:
    """The oracle arm: the headline workload (same configuration, metric and unit as the GPU arm):
    the oracle builds the 256 x 256 H^2 once (set-up, timed and reported), then every step
    applies its matvec to nrhs 1, 32 and 256 right-hand sides; rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O

    p, b = CFG["problem"], CFG["build"]
    N = p.N
    mask = W.sensor_mask(N, p.m, p.sensor_seed)
    op = O.HeatHessian(p.n, p.kappa, p.T, p.sigma, mask)
    t0 = time.perf_counter()
    h, res = O.build(op, W.grid_coords(p.n), b.leaf, b.adm, b.eta, b.tol, b.kmax, b.q0, b.b_inc, b.q_max,
                     b.adaptive, b.seed, certified=HEADLINE_CERTIFIED)
    build_s = time.perf_counter() - t0
    ent = O.storage_entries(h)
    st = {"entries_D": ent["D"], "entries_S": ent["S"], "entries_U": ent["U"], "entries_E": ent["E"]}
    Xs = {nr: W.rhs(N, nr, CFG["rhs_seed"] + nr) for nr in CFG["nrhs"]}

    def step():
        by, tt = 0.0, 0.0
        for nr, X in Xs.items():
            t0 = time.perf_counter()
            O.matvec(h, X)
            tt += time.perf_counter() - t0
            by += matvec_bytes(st, N, nr)
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
    dump = os.path.join(tempfile.gettempdir(), f"h2bench_ref_{os.getpid()}.npz")
    side = {}
    try:
        r, U, E, S, D = O.factor_arrays(h)
        np.savez(dump, ranks=r, U=U, E=E, S=S, D=D)
        side = oracle_side_measurements(None, dump)
    except Exception as e:   # the side measurements are context; the arm's value stands without them
        side = {"side_measurements_failed": str(e)[-300:]}
    finally:
        if os.path.exists(dump):
            os.remove(dump)
    sample = (f"oracle matvec (nrhs {list(CFG['nrhs'])}) of the oracle-built H^2 of the headline workload "
              f"({CFG['name']}, N={N}) per step; the oracle construction (set-up) took {build_s:.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(CFG),
            "cpu_baseline": {"value": val, "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample, "build_s": build_s, "samples": int(res.samples - res.norm_its),
                             **side},
            "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(cfg: dict) -> dict:
    p, b = cfg["problem"], cfg["build"]
    return {"workload": cfg["name"], "N": p.N, "grid": f"{p.n}x{p.n}", "sensors": p.m, "kappa": p.kappa,
            "leaf": b.leaf, "adm": "strong", "eta": b.eta, "kmax": b.kmax, "tol": b.tol,
            "range_bases": "certified" if HEADLINE_CERTIFIED else "all probes",
            "nrhs": list(cfg["nrhs"]), "mode": "FP64",
            "l2": "H2 factors larger than L2 (no flush needed)", "parallelism": "replicas"}


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
    ap.add_argument("--no-update", action="store_true")
    ap.add_argument("--no-sampling", action="store_true")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--no-advdiff", action="store_true")
    ap.add_argument("--no-certified", action="store_true")
    ap.add_argument("--n", type=int, default=None,
                    help="grid size of the stepped Hessian (profiling captures on smaller cases; bench lines use the default)")
    ap.add_argument("--precision-n", type=int, default=512, help="grid size of the precision section")
    ap.add_argument("--oracle-worker", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_worker is not None:
        print(json.dumps(oracle_worker(json.loads(args.oracle_worker))), flush=True)
        return
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
        cpu = cpu_baseline_full()

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
                           seed=b.seed, stream=stream, certified=int(HEADLINE_CERTIFIED))
    nrhs_list = list(CFG["nrhs"])
    Xd = {nr: torch.from_numpy(np.ascontiguousarray(W.rhs(N, nr, CFG["rhs_seed"] + nr).T)).cuda()
          for nr in nrhs_list}
    Yd = {nr: torch.empty_like(Xd[nr]) for nr in nrhs_list}

    nr_roof = max(nrhs_list)

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
            # per-stage events (on this stream) around the widest matvec: the roofline's kernel
            G.profile(nr == nr_roof)
            a.record(stream)
            G.matvec(Xd[nr], Yd[nr], nr, h2.H2_FP64, stream=stream)
            c.record(stream)
            G.profile(False)
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
    gemm_ms, gemm_flops, gemm_n, gemm_bytes = h2.gemm_profile_read()
    stack_prof = [h2.stack_profile_read(w) for w in (0, 1)]
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

    fp64_meas = fp64_peak_measured(torch, stream)
    # roofline of the metric's dominant kernel: the FP64 gather kernel of the leaf expansion and
    # near field (mv_leaf_near_kernel) in the nrhs = 256 matvec, timed with per-stage CUDA events on
    # the matvec's stream inside the timed steps; algorithmic flops of that stage: every stored
    # off-diagonal near block applied twice (D and D^T), every diagonal block once, plus U_t yh_t
    _, sizes = tree.boxes(tree.L)
    stage_ms = {}
    for G, _, _ in results:
        for k, (ms, nl) in G.profile_read().items():
            if nl:
                stage_ms.setdefault(k, []).append(ms)
    ln_ms = float(np.mean(stage_ms["leaf_near"]))
    ln_flops = near_flops(st, sizes, nr_roof) + 2.0 * nr_roof * st["entries_U"]
    ln_tf = ln_flops / (ln_ms / 1e3) / 1e12
    ln_alg_bytes = st["entries_D"] * 8 + 2 * N * nr_roof * 8
    roofline = {"bound": "alu", "achieved": ln_tf, "peak": fp64_meas, "unit": "TFLOP/s",
                "frac": ln_tf / fp64_meas,
                "traffic": MATVEC_TRAFFIC_SMALL["dram_bytes"] * ln_alg_bytes / MATVEC_TRAFFIC_SMALL["algorithmic_bytes"],
                "kernel": f"mv_leaf_near_kernel (FP64 gather: near field + leaf expansion, nrhs={nr_roof})",
                "peak_source": "measured: cuBLAS DGEMM 4096^3 (torch.matmul float64) on this GPU, best of 5",
                "flops_per_launch": ln_flops, "ms_per_launch": ln_ms,
                "stage_ms": {k: float(np.mean(v)) for k, v in stage_ms.items()},
                "fp64_peak_derived_TFLOPs": fp64,
                "algorithmic_bytes_per_launch": ln_alg_bytes,
                "traffic_note": "DRAM read+write bytes per launch: ncu capture at %s (%.3e B for %.3e algorithmic B), "
                                "scaled by the algorithmic bytes; each CTA (leaf, right-hand-side tile) re-reads the "
                                "leaf's near blocks" % (MATVEC_TRAFFIC_SMALL["grid"], MATVEC_TRAFFIC_SMALL["dram_bytes"],
                                                         MATVEC_TRAFFIC_SMALL["algorithmic_bytes"])}
    # the construction's FP64 batched GEMM (operator DSTs, piece subtraction, stacked-QR inputs),
    # timed per launch with events on the build stream over the timed steps
    gemm_tf = gemm_flops / (gemm_ms / 1e3) / 1e12 if gemm_ms > 0 else None
    roofline_build_gemm = {"bound": "alu", "achieved": gemm_tf, "peak": fp64_meas, "unit": "TFLOP/s",
                           "frac": (gemm_tf / fp64_meas) if gemm_tf else None, "traffic": None,
                           "kernel": "gemm_tiles_kernel (FP64 batched GEMM of the construction)",
                           "peak_source": "measured: cuBLAS DGEMM (as roofline)",
                           "launches": gemm_n, "ms": gemm_ms,
                           "flops_per_launch": gemm_flops / max(gemm_n, 1), "ms_per_launch": gemm_ms / max(gemm_n, 1),
                           "algorithmic_bytes_per_launch": gemm_bytes / max(gemm_n, 1),
                           "traffic_note": "per-launch DRAM bytes vary with the problem list; sampled launches "
                                           "in profiles/gemm_tiles_n128_n256.md"}
    # the recompression's stacked Householder QR and truncated SVD (FP64-pipe bound), timed with
    # events over the timed steps (the stacked QR per pass: its width classes run concurrently on
    # side streams, one span from the fork to the join); flops are those of their QR
    # factorisations only
    roofline_build_stacked = {}
    for name, (ms, fl, n) in zip(("stacked_r_kernel", "stacked_svd_kernel"), stack_prof):
        tf = fl / (ms / 1e3) / 1e12 if ms > 0 else None
        roofline_build_stacked[name] = {"bound": "alu", "achieved": tf, "peak": fp64_meas, "unit": "TFLOP/s",
                                        "frac": (tf / fp64_meas) if tf else None, "launches": n,
                                        "ms_per_step": ms / args.steps, "qr_flops_per_step": fl / args.steps}
    # FP64 near field at nrhs = 1 (the atomic scatter kernel), outside the timed region
    Gp = results[-1][0]
    Gp.profile(True)
    for _ in range(5):
        Gp.matvec(Xd[1], Yd[1], 1, h2.H2_FP64, stream=stream)
    prof = Gp.profile_read()
    Gp.profile(False)
    nr_ms, nr_n = prof["near"]
    nr_s = nr_ms / nr_n / 1e3
    achieved = near_flops(st, sizes, 1) / nr_s / 1e12
    roofline_matvec_nrhs1 = {"bound": "alu", "achieved": achieved, "peak": fp64_meas, "unit": "TFLOP/s",
                             "frac": achieved / fp64_meas, "traffic": None,
                             "kernel": "mv_scatter_kernel<double,...,1,true> (near field, nrhs=1)",
                             "peak_source": "measured: cuBLAS DGEMM (as roofline)",
                             "hbm_GBps": st["entries_D"] * 8 / nr_s / 1e9}
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

    # end to end through the public C-ABI call with HOST buffers (h2_matvec_host: pinned host X and
    # Y, host-to-device copy, matvec, device-to-host copy inside the call and the timed region)
    Gp2 = results[-1][0]
    Xh = {nr: torch.empty((nr, N), dtype=torch.float64, pin_memory=True) for nr in nrhs_list}
    Yh = {nr: torch.empty((nr, N), dtype=torch.float64, pin_memory=True) for nr in nrhs_list}
    for nr in nrhs_list:
        Xh[nr].copy_(Xd[nr].cpu())
    for nr in nrhs_list:      # warm-up: staging buffers grown, graphs captured
        Gp2.matvec_host(Xh[nr], Yh[nr], nr, h2.H2_FP64, stream=stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = 3
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        for nr in nrhs_list:
            Gp2.matvec_host(Xh[nr], Yh[nr], nr, h2.H2_FP64, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_s = e0.elapsed_time(e1) / 1e3
    e2e_bytes = reps * sum(by[nr] for nr in nrhs_list)
    e2e = {"value": aggregate_throughput(e2e_bytes, e2e_s, dist) / 1e9, "unit": "GB/s",
           "h2d_bytes_per_step": sum(N * nr * 8 for nr in nrhs_list),
           "d2h_bytes_per_step": sum(N * nr * 8 for nr in nrhs_list),
           "call": "h2_matvec_host (C ABI, pinned host buffers)"}

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

    small = None
    if rank == 0 and not args.no_small:
        small = small_section(h2, torch, stream)

    sampling = None
    if rank == 0 and not args.no_sampling:
        sampling = sampling_section(h2, torch, stream)

    update = None
    if rank == 0 and not args.no_update:
        update = update_section(h2, torch, stream, Gp2, N, float(np.mean(build_ms)) / 1e3)

    certified = None
    if rank == 0 and not args.no_certified:
        certified = certified_section(h2, torch, stream)

    inversion = None
    if rank == 0 and not args.no_inversion:
        inversion = inversion_section(h2, torch, stream)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(CFG),
            "build_s": float(np.mean(build_ms)) / 1e3,
            "rel_err_2norm": rel_err,
            "samples": st["samples"], "norm_products": st["norm_products"], "max_rank": st["max_rank"],
            "range_probes": st["range_probes"], "proj_probes": st["proj_probes"],
            "matvec_ms": {str(nr): float(np.mean(mv_ms[nr])) for nr in nrhs_list},
            "matvec_GBps": {str(nr): by[nr] / (np.mean(mv_ms[nr]) / 1e3) / 1e9 for nr in nrhs_list},
            "stored_bytes_fp64": (st["entries_D"] + st["entries_S"] + st["entries_U"] + st["entries_E"]) * 8,
            "hbm_view": hbm_view,
            "roofline": roofline, "roofline_build_gemm": roofline_build_gemm,
            "roofline_build_stacked": roofline_build_stacked,
            "roofline_matvec_nrhs1": roofline_matvec_nrhs1,
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
        if update is not None:
            line["lowrank_update"] = update
        if sampling is not None:
            line["sampling_structure"] = sampling
        if small is not None:
            line["small_n32"] = small
        if certified is not None:
            line["certified_bases"] = certified
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    for G, _, _ in results:
        G.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
