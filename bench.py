#!/usr/bin/env python
"""Benchmark of the compression hot path on one GB300 (or N replicas).

Workload (the metric's configuration): HBS-ID compression at tol 1e-7 of the
FP32 log-kernel matrix of N = 65536 points on the ellipse (cos t, 0.5 sin t),
leaves of 256 points, r = 60 random vectors per level and side, applied as a
dense black box by the library's sampling GEMM.  One step = one full
hm_compress_hbs call (all levels, the diagonal probe and the HBS-ID sweep) with
the 17.2 GB operator resident in HBM.  The operator is larger than L2, so no
extra flush is needed between steps.

Headline precision: HM_A32 (the FP32 operator applied to FP64 blocks by the
exact-accumulation split GEMM on the tensor cores, FP64 peeling, bases and
ID), the configuration that meets rel err <= 1e-7 at this size; its Frobenius
error against the operator is measured after the timed steps.  The HM_MIXED
(FP32 samples and bases) compression is timed beside it.

Also reported: the HODLR adjoint workload (N = 262144, k = 32, leaves of 256,
forward apply + hand-written adjoint per step), the roofline of the dominant
kernel (the sampling GEMM), nvidia-smi clocks sampled during the timed region,
an end-to-end number through the C ABI with the operator copied from pinned
host memory every step, and the FP64 CPU oracle timed on a bounded sample.

`--impl reference` times the CPU oracle instead (the reference arm).
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
sys.path.insert(0, ROOT)

METRIC = "compress ms at N=65536 (rel err ≤1e-7), % of roofline; HODLR adjoint applies/s"
N_HEAD, LEAF_HEAD, R_HEAD, TOL_HEAD = 65536, 256, 60, 1e-7
N_ADJ, LEAF_ADJ, K_ADJ = 262144, 256, 32
ORACLE_SAMPLE_N = 8192
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--n", type=int, default=N_HEAD, help="operator size (default: the metric's)")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-adjoint", action="store_true")
    ap.add_argument("--skip-frob", action="store_true", help="skip the full Frobenius error check")
    ap.add_argument("--skip-mixed", action="store_true", help="skip the HM_MIXED comparison run")
    ap.add_argument("--skip-fp64", action="store_true", help="skip the HM_FP64 comparison run")
    ap.add_argument("--skip-batched", action="store_true", help="skip the batched many-operator run")
    ap.add_argument("--skip-matrix-free", action="store_true",
                    help="skip the matrix-free log-kernel runs")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for key in ("hbm_gbs", "hbm_GBs", "hbm"):
                if key in d:
                    return float(d[key]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def time_events(fn, reps, torch):
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


# DRAM traffic of one k_gemm_esg launch from an ncu capture of a level-0 sample
# (60 columns, half of K active) at N = 16384: 541.4 MB read + 3.1 MB written for
# 552.6 MB of algorithmic bytes.  Traffic grows with the units processed (rows x
# active K; a split over K gives each block a disjoint share of the windows), so a
# launch at another N moves this ratio times its own algorithmic bytes.
ESG_TRAFFIC_PER_ALG_BYTE = (541.4e6 + 3.1e6) / (4.0 * 16384 * 8192 + 16.0 * 16384 * 60)


def gemm_roofline(hm, torch, A, op, tree, n, peak_gbs, peak_kind):
    """Dominant HBM-bound kernel: one black-box call with a level-0 test matrix half
    (Y_1 = A Omega_2, Omega_2 nonzero on the right child's rows only), FP64 block."""
    r = R_HEAD
    X = torch.empty((2 * r, n), device=A.device, dtype=torch.float64)
    hm.hm_gaussian_test_matrix(tree, 0, r, 2, hm.HM_A32, X)
    Xh = X[:r]
    Y = torch.empty_like(Xh)
    call = lambda: hm.hm_dense_apply(op, 0, Xh, Y)  # noqa: E731
    for _ in range(2):
        call()
    ms = time_events(call, 5, torch)
    k_active = n - tree.node(2)[1]  # rows of Omega_2's support: the right child
    alg_bytes = 4.0 * n * k_active + 8.0 * n * r * 2
    gbs = alg_bytes / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak_gbs, "unit": "GB/s",
            "frac": round(gbs / peak_gbs, 4), "traffic": round(alg_bytes * ESG_TRAFFIC_PER_ALG_BYTE),
            "traffic_source": "ncu dram read+write of the same launch at N=16384, scaled by the "
                              "algorithmic bytes (rows x active K)",
            "kernel": "k_gemm_esg (exact-accumulation split sampling GEMM, A Omega_2 at level 0)",
            "algorithmic_bytes_per_launch": alg_bytes, "launch_ms": round(ms, 4),
            "peak_source": f"{peak_kind} HBM copy bandwidth",
            "note": "launch_ms covers hm_dense_apply: the X pre-cut kernel and the GEMM"}


def bf16_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return float(json.load(open(p))["bf16_tflops"]), "measured"
        except Exception:
            pass
    return 1900.0, "fallback"


def matrix_free_bench(hm, torch, dev, steps, n, big_n):
    """The headline compression with the matrix-free log-kernel black box (entries
    formed in the sampling GEMM from two tables, no operator in HBM), its GEMM
    against the tensor roofline, and one compression at big_n (twice the headline
    size) with its error estimated on 64 sampled rows."""
    import numpy as np
    op = hm.hm_log_kernel_operator_create(n)
    tree = hm.Tree(n, LEAF_HEAD)
    kw = dict(tol=TOL_HEAD, r=R_HEAD, seed=2, prec=hm.HM_A32, hbs_id=1)
    h = hm.hm_compress_hbs(op, tree, **kw)
    del h
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        h = hm.hm_compress_hbs(op, tree, **kw)
        if _ < steps - 1:
            del h
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    Wv = torch.randn((10, n), device=dev, generator=torch.Generator(device=dev).manual_seed(11),
                     dtype=torch.float64)
    Wv /= Wv.norm(dim=1, keepdim=True)
    Yt, Yc = torch.empty_like(Wv), torch.empty_like(Wv)
    hm.hm_dense_apply(op, 0, Wv, Yt)
    hm.hm_apply(h, 0, Wv, Yc)
    torch.cuda.synchronize()
    E = float(((Yt - Yc).norm(dim=1) / Yt.norm(dim=1)).max())
    # one level-0 black-box call (Y_1 = A Omega_2): 10 slice products of the
    # active half of K against 64 (60 used) columns on the tensor cores
    r = R_HEAD
    X = torch.empty((2 * r, n), device=dev, dtype=torch.float64)
    hm.hm_gaussian_test_matrix(tree, 0, r, 2, hm.HM_A32, X)
    Xh = X[:r]
    Y = torch.empty_like(Xh)
    call = lambda: hm.hm_dense_apply(op, 0, Xh, Y)  # noqa: E731
    for _ in range(2):
        call()
    cms = time_events(call, 5, torch)
    k_active = n - tree.node(2)[1]
    flops = 10.0 * 2.0 * n * k_active * 64
    peak, kind = bf16_peak()
    tf = flops / (cms * 1e-3) / 1e12
    out = {"ms": round(ms, 3), "estimate_E": E, "ranks": [h.info["min_rank"], h.info["max_rank"]],
           "saturated": h.info["saturated"], "t_blackbox_ms": round(h.info["t_blackbox_ms"], 3),
           "operator_bytes_in_hbm": 12 * n,
           "gemm": {"bound": "tensor", "kernel": "k_gemm_esg<0,1> (entries generated in the cutter "
                                                  "warps)",
                    "achieved": round(tf, 1), "peak": peak, "unit": "TFLOP/s",
                    "frac": round(tf / peak, 4), "launch_ms": round(cms, 4),
                    "algorithmic_flops_per_launch": flops,
                    "peak_source": f"{kind} dense bf16 (burst)",
                    "definition": "10 BF16 slice products x 2 x rows x active K x 64 columns"}}
    del h, op
    if big_n:
        opb = hm.hm_log_kernel_operator_create(big_n)
        rows = torch.randperm(big_n, generator=torch.Generator().manual_seed(8))[:64].sort().values
        Ar = torch.empty((64, big_n), device=dev, dtype=torch.float32)
        for q, i in enumerate(rows.tolist()):
            hm.hm_log_kernel_entries(opb, i, i + 1, 0, big_n, Ar[q:q + 1])
        Eb = torch.zeros((64, big_n), device=dev, dtype=torch.float64)
        Eb[torch.arange(64), rows.to(dev)] = 1.0

        def sampled_err(h):
            Rc = torch.empty_like(Eb)
            hm.hm_apply(h, 1, Eb, Rc)
            torch.cuda.synchronize()
            return float((Rc - Ar.double()).norm() / Ar.double().norm())
        treeb = hm.Tree(big_n, LEAF_HEAD)
        res = {}
        for name, fn, kwb in (("hodlr", hm.hm_compress_hodlr, dict(tol=1e-8, r=100, seed=2,
                                                                    prec=hm.HM_A32)),
                              ("hbsid", hm.hm_compress_hbs, dict(kw, r=64))):
            eb0, eb1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            eb0.record()
            hb = fn(opb, treeb, **kwb)
            eb1.record()
            torch.cuda.synchronize()
            res[name] = {"ms": round(eb0.elapsed_time(eb1), 2), "rel_frob_err_sampled": sampled_err(hb),
                         "tol": kwb["tol"], "r": kwb["r"],
                         "ranks": [hb.info["min_rank"], hb.info["max_rank"]],
                         "saturated": hb.info["saturated"]}
            del hb
        res["note"] = ("one compression each; relative Frobenius error on 64 sampled rows against the "
                       "operator's entries; the FP32 rounding of the entries leaves a floor of about "
                       "sqrt(L) x 3.4e-8 (1.0e-7 at L = 9) that no tolerance goes below")
        res["fp32_noise_floor"] = float(np.sqrt(treeb.levels) * 2.0 ** -24 / np.sqrt(3.0))
        out["n%d" % big_n] = res
        del opb
    return out


def adjoint_bench(hm, torch, dev, steps, warmup):
    import numpy as np
    n, m, k = N_ADJ, LEAF_ADJ, K_ADJ
    tree = hm.Tree(n, m)
    L = tree.levels
    g = torch.Generator(device=dev).manual_seed(5)
    U = torch.randn((L, k, n), device=dev, generator=g)
    V = torch.randn((L, k, n), device=dev, generator=g)
    D = torch.randn((1 << L, m, m), device=dev, generator=g)
    D += float(n) * torch.eye(m, device=dev)
    x = torch.randn(n, device=dev, generator=torch.Generator(device=dev).manual_seed(6))
    b = torch.randn(n, device=dev, generator=torch.Generator(device=dev).manual_seed(7))
    y = torch.empty_like(x)
    r = torch.empty_like(x)
    gx, gU, gV, gD = (torch.empty_like(t) for t in (x, U, V, D))

    def step():  # the fused training step: y = H x, r = y - b, gradients at r
        hm.hm_hodlr_factored_loss_grad(tree, k, U, V, D, x, b, 2.0, y, r, gx, gU, gV, gD)

    def step_two_calls():  # the same through the separate forward and adjoint calls
        hm.hm_hodlr_factored_apply(tree, k, U, V, D, x, y)
        torch.sub(y, b, out=r)
        hm.hm_hodlr_factored_adjoint(tree, k, U, V, D, x, r, 2.0, gx, gU, gV, gD)
    for _ in range(warmup):
        step()
        step_two_calls()
    ms2 = time_events(step_two_calls, steps, torch)
    ms_eager = time_events(step, steps, torch)
    # the same call captured once in a CUDA graph and replayed per step, as a
    # training loop runs it (stream-ordered scratch and the counter clear are
    # graph nodes; no launch gaps between the step's kernels)
    ms_graph, graph_note = None, None
    try:
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            step()
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, capture_error_mode="thread_local"):
            step()
        for _ in range(warmup):
            graph.replay()
        ms_graph = time_events(graph.replay, steps, torch)
    except Exception as exc:  # report, and keep the eager number
        graph_note = f"capture failed: {exc!r}"[:200]
    ms = ms_eager
    fbytes = 4.0 * (U.numel() + V.numel() + D.numel())
    moved = 2 * fbytes + fbytes + 4.0 * n * 8  # read factors twice, write gradients once
    peak, kind = peaks()
    frac = lambda t: round(moved / (t * 1e-3) / 1e9 / peak, 4)  # noqa: E731
    return {"value": round(1000.0 / ms, 2), "unit": "(forward + adjoint) applies/s",
            "ms_per_apply_pair": round(ms, 4), "config": {"n": n, "k": k, "leaf": m, "levels": L},
            "bytes_per_pair": moved, "achieved_GBs": round(moved / (ms * 1e-3) / 1e9, 1),
            "frac": frac(ms), "peak_GBs": peak,
            "path": "hm_hodlr_factored_loss_grad (forward, residual and adjoint in one call), "
                    "called per step",
            "graph": {"ms_per_apply_pair": None if ms_graph is None else round(ms_graph, 4),
                      "frac": None if ms_graph is None else frac(ms_graph),
                      "path": "the same call captured once in a CUDA graph, replayed per step",
                      "note": graph_note},
            "two_calls": {"ms_per_apply_pair": round(ms2, 4), "frac": frac(ms2),
                          "path": "hm_hodlr_factored_apply + torch.sub + hm_hodlr_factored_adjoint"},
            "bytes_definition": "factors U, V, D read by the forward apply and by the adjoint, "
                                "their gradients written once, x / b / y / gx vectors"}


def batched_bench(hm, torch, dev, count=64):
    """Batched workload: 64 independent synthetic HODLR operators (N log-uniform in [2048, 32768]
    rounded to 64, k uniform in [8, 40], leaves of 64, r = k + 10), each formed densely in
    FP32 on the device from its seeded factors, compressed by one hm_compress_batched call
    in HM_A32 (FP64 pipeline, tensor-core products)."""
    import numpy as np
    import workloads as W
    specs = W.batched_hodlr_specs(count)
    mats, ops, trees, opts = [], [], [], []
    for sp in specs:
        N, k = sp["N"], sp["k"]
        f = W.synthetic_hodlr_factors(N, 64, k, seed=sp["op_seed"], shift=float(N), dtype=np.float32)
        A = torch.zeros((N, N), device=dev, dtype=torch.float32)
        st, sz = f["start"], f["size"]
        for j in range(1, f["L"] + 1):
            Uj = torch.from_numpy(f["U"][j]).to(dev)
            Vj = torch.from_numpy(f["V"][j]).to(dev)
            for a in range(2 ** j, 2 ** (j + 1)):
                b = a ^ 1
                A[st[a]:st[a] + sz[a], st[b]:st[b] + sz[b]] = Uj[st[a]:st[a] + sz[a]] @ Vj[st[b]:st[b] + sz[b]].T
        for i, t in enumerate(range(2 ** f["L"], 2 ** (f["L"] + 1))):
            A[st[t]:st[t] + sz[t], st[t]:st[t] + sz[t]] = torch.from_numpy(f["D"][i]).to(dev)
        mats.append(A)
        ops.append(hm.hm_dense_operator_create(A, fp64_blocks=True, tensor_cores=True))
        trees.append(hm.Tree(N, 64))
        opts.append(dict(k=k, p=10, seed=sp["omega_seed"], prec=hm.HM_A32))
    # the concurrency (streams of the level-synchronous batch) picked by the
    # library's autotuner from timed runs of this batch; the handles do not depend on it
    cands = (4, 8, 16)
    best, tune_ms = hm.hm_tune_batched(ops, trees, "hodlr", opts, candidates=cands)
    hs = hm.hm_compress_batched(ops, trees, "hodlr", opts, max_concurrency=best)  # warm-up
    del hs
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hs = hm.hm_compress_batched(ops, trees, "hodlr", opts, max_concurrency=best)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3
    errs = []
    g = torch.Generator(device=dev).manual_seed(12)
    for A, h, op in zip(mats, hs, ops):
        N = A.shape[0]
        W4 = torch.randn((4, N), device=dev, dtype=torch.float64, generator=g)
        Yt, Yc = torch.empty_like(W4), torch.empty_like(W4)
        hm.hm_dense_apply(op, 0, W4, Yt)
        hm.hm_apply(h, 0, W4, Yc)
        errs.append(float(((Yt - Yc).norm(dim=1) / Yt.norm(dim=1)).max()))
    ns = [sp["N"] for sp in specs]
    return {"ops": count, "ms": round(ms, 2), "compressions_per_s": round(count / (ms * 1e-3), 2),
            "n_range": [min(ns), max(ns)], "k_range": [min(sp["k"] for sp in specs), max(sp["k"] for sp in specs)],
            "max_estimate_E": max(errs), "precision": "HM_A32",
            "autotune": {"candidates": list(cands), "ms": tune_ms, "chosen": best,
                         "by": "hm_tune_batched (one timed batch per candidate concurrency)"},
            "note": "host wall time of one hm_compress_batched call (all operators resident)"}


def oracle_sample(n_sample: int):
    """The FP64 oracle on a bounded sample of the headline workload."""
    import numpy as np
    import workloads as W
    from oracle import hbs as ohbs
    from oracle import hodlr as ohodlr
    from oracle.tree import build_tree
    A = W.log_kernel(n_sample)
    t0 = time.time()
    h = ohbs.compress(ohodlr.dense_apply_fn(A), build_tree(n_sample, LEAF_HEAD), r=R_HEAD, seed=2,
                      mixed=True)
    ohbs.to_hbsid(h, tol=TOL_HEAD)
    return time.time() - t0


def cpu_baseline_line():
    """The oracle timed on a bounded sample: the same workload at N = 8192 (the
    full N = 65536 run would take minutes of host time).  `value` is the measured
    sample time; the N^2 extrapolation to the headline size is a separate field."""
    cores = len(os.sched_getaffinity(0))
    secs = oracle_sample(ORACLE_SAMPLE_N)
    scale = (N_HEAD / ORACLE_SAMPLE_N) ** 2
    return {"value": round(secs * 1e3, 1), "unit": "ms", "cores": cores, "kind": "oracle",
            "n": ORACLE_SAMPLE_N,
            "sample": (f"FP64 NumPy oracle, HBS + HBS-ID compression of the same log-kernel "
                       f"workload at N={ORACLE_SAMPLE_N} (leaves {LEAF_HEAD}, r={R_HEAD}, "
                       f"tol 1e-7), one run on {cores} host cores"),
            "extrapolated_to_n65536_ms": round(secs * scale * 1e3, 1),
            "extrapolation": f"x (65536/{ORACLE_SAMPLE_N})^2: the dense black box, which "
                             "dominates the oracle, grows as N^2 (an estimate, not a measurement)"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    cores = len(os.sched_getaffinity(0))
    for _ in range(args.warmup):
        oracle_sample(2048)
    times = [oracle_sample(ORACLE_SAMPLE_N) for _ in range(args.steps)]
    secs = statistics.median(times)
    val = secs * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": round(val, 1), "unit": "ms",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(val, 1), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"HBS-ID compression, log kernel on ellipse, N={ORACLE_SAMPLE_N} "
                                   f"(bounded sample of the N=65536 workload), leaves 256, tol 1e-7, "
                                   "r=60", "n": ORACLE_SAMPLE_N, "leaf": LEAF_HEAD, "tol": TOL_HEAD,
                       "r": R_HEAD},
            "cpu_baseline": {"value": round(val, 1), "unit": "ms", "cores": cores, "kind": "oracle",
                             "n": ORACLE_SAMPLE_N,
                             "sample": f"FP64 NumPy oracle at N={ORACLE_SAMPLE_N}, median of "
                                       f"{args.steps} steps",
                             "extrapolated_to_n65536_ms": round(val * (N_HEAD / ORACLE_SAMPLE_N) ** 2, 1),
                             "extrapolation": f"x (65536/{ORACLE_SAMPLE_N})^2 (an estimate, not a "
                                              "measurement)"},
            "e2e": {"value": round(val, 1), "unit": "ms", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch
    import paper_1503_07152_gb300 as hm
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    n = args.n
    peak_gbs, peak_kind = peaks()
    A = torch.empty((n, n), device=dev, dtype=torch.float32)
    hm.hm_gen_log_kernel(A)
    torch.cuda.synchronize()
    op = hm.hm_dense_operator_create(A, fp64_blocks=True, tensor_cores=True)
    tree = hm.Tree(n, LEAF_HEAD)
    kw = dict(tol=TOL_HEAD, r=R_HEAD, seed=2, prec=hm.HM_A32, hbs_id=1)

    def step():
        return hm.hm_compress_hbs(op, tree, **kw)
    for _ in range(args.warmup):
        h = step()
    del h
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = hm.hm_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    infos = []
    for _ in range(args.steps):
        h = step()
        infos.append(h.info)
        if _ < args.steps - 1:
            del h
    ev1.record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = (hm.hm_launch_count() - l0) // args.steps
    ms = ev0.elapsed_time(ev1) / args.steps
    clk = clocks.stop()
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = ms / ws
    # accuracy of the last compression (outside the timed region): the relative
    # Frobenius error against the FP32 operator over all N^2 entries, and a
    # 10-vector estimate
    err = None if args.skip_frob else hm.hm_rel_frob_error(h, A)
    Wv = torch.randn((10, n), device=dev, generator=torch.Generator(device=dev).manual_seed(11),
                     dtype=torch.float64)
    Wv /= Wv.norm(dim=1, keepdim=True)
    Yt = torch.empty_like(Wv)
    Yc = torch.empty_like(Wv)
    hm.hm_dense_apply(op, 0, Wv, Yt)
    hm.hm_apply(h, 0, Wv, Yc)
    torch.cuda.synchronize()
    E = float(((Yt - Yc).norm(dim=1) / Yt.norm(dim=1)).max())
    # the same compression with in-order sampling (no look-ahead stream), outside
    # the timed region: the look-ahead's share of the step time
    kw_io = dict(kw, lookahead=-1)
    hm.hm_compress_hbs(op, tree, **kw_io)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps_io = max(1, min(3, args.steps))
    e0.record()
    for _ in range(reps_io):
        h_io = hm.hm_compress_hbs(op, tree, **kw_io)
    e1.record()
    torch.cuda.synchronize()
    in_order = {"ms": round(e0.elapsed_time(e1) / reps_io, 3),
                "t_blackbox_ms": round(h_io.info["t_blackbox_ms"], 3),
                "note": "hm_opts.lookahead = -1: every black-box product on the compression "
                        "stream; the timed steps sample the next level's A-side block on a "
                        "second stream while the current level's panels are factored"}
    del h_io
    # the FP32-sample compression beside it
    mixed = None
    if not args.skip_mixed:
        opm = hm.hm_dense_operator_create(A)
        kwm = dict(kw, prec=hm.HM_MIXED)
        hm_ = hm.hm_compress_hbs(opm, tree, **kwm)
        del hm_
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        hm_ = hm.hm_compress_hbs(opm, tree, **kwm)
        e1.record()
        torch.cuda.synchronize()
        Wf = Wv.float()
        Ytf, Ycf = torch.empty_like(Wf), torch.empty_like(Wf)
        hm.hm_dense_apply(opm, 0, Wf, Ytf)
        hm.hm_apply(hm_, 0, Wf, Ycf)
        torch.cuda.synchronize()
        mixed = {"ms": round(e0.elapsed_time(e1), 3), "precision": "HM_MIXED (FP32 samples and bases)",
                 "estimate_E": float(((Ytf - Ycf).norm(dim=1) / Ytf.norm(dim=1)).max()),
                 "t_blackbox_ms": round(hm_.info["t_blackbox_ms"], 3),
                 "ranks": [hm_.info["min_rank"], hm_.info["max_rank"]]}
        del hm_, opm
    # the all-FP64 compression beside it: the same FP32 entries widened to an FP64
    # operator (34 GB at N=65536), FP64 black box on the CUDA cores; one run
    fp64 = None
    if not args.skip_fp64:
        A64 = A.double()
        op64 = hm.hm_dense_operator_create(A64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        h64 = hm.hm_compress_hbs(op64, tree, **dict(kw, prec=hm.HM_FP64))
        e1.record()
        torch.cuda.synchronize()
        Yt64, Yc64 = torch.empty_like(Wv), torch.empty_like(Wv)
        hm.hm_dense_apply(op64, 0, Wv, Yt64)
        hm.hm_apply(h64, 0, Wv, Yc64)
        torch.cuda.synchronize()
        fp64 = {"ms": round(e0.elapsed_time(e1), 3),
                "precision": "HM_FP64 (FP64 operator holding the same FP32 entries, FP64 black box "
                             "on the CUDA cores, FP64 samples, bases and ID)",
                "estimate_E": float(((Yt64 - Yc64).norm(dim=1) / Yt64.norm(dim=1)).max()),
                "t_blackbox_ms": round(h64.info["t_blackbox_ms"], 3),
                "ranks": [h64.info["min_rank"], h64.info["max_rank"]],
                "note": "one run without warm-up, outside the timed region"}
        del h64, op64, A64, Yt64, Yc64
        torch.cuda.empty_cache()
    roof = gemm_roofline(hm, torch, A, op, tree, n, peak_gbs, peak_kind)
    info = infos[-1]
    # the whole compression against the HBM roofline: the two black-box calls of a
    # level and side each read the half of A where their test matrix is nonzero
    # (one full read of A per level and side), the identity probe reads it once
    # more, and every call moves its FP64 sample blocks in and out; the bases, peel
    # and factorizations move about 1 GB more, left out of the algorithmic bytes
    reads_A = 2 * tree.levels + 1
    comp_bytes = reads_A * 4.0 * n * n + 16.0 * n * (info["cols_A"] + info["cols_At"])
    comp_gbs = comp_bytes / (ms * 1e-3) / 1e9
    roof["compression"] = {
        "algorithmic_bytes": comp_bytes, "achieved": round(comp_gbs, 1),
        "frac": round(comp_gbs / peak_gbs, 4), "floor_ms": round(comp_bytes / peak_gbs / 1e6, 2),
        "definition": f"{reads_A} reads of the FP32 operator (one per level and side, one for the "
                      "identity probe) + 16 B per sample entry of every black-box call, divided by "
                      "ms_per_step"}
    roof["compression_frac"] = roof["compression"]["frac"]
    # per-phase device time of one more (profiled) compression, outside the timed region
    hm.hm_set_profiling(True)
    hp = step()
    hm.hm_set_profiling(False)
    segs = hm.hm_profile(hp)
    del hp
    phase_ms = {}
    for sg in segs:
        phase_ms[sg["phase"]] = phase_ms.get(sg["phase"], 0.0) + sg["ms"]
    per_level = {}
    for sg in segs:
        key = f"L{sg['level']}{'AT' if sg['side'] else 'A'}"
        per_level.setdefault(key, {})
        per_level[key][sg["phase"]] = round(per_level[key].get(sg["phase"], 0.0) + sg["ms"], 2)
    phases = {"total_ms": {k_: round(v, 2) for k_, v in phase_ms.items()}, "per_level": per_level,
              "note": "CUDA-event segments of one profiled compression (hm_set_profiling); level L "
                      "side A is the identity probe"}
    bb_share = info["t_blackbox_ms"] / info["t_compress_ms"] if info["t_compress_ms"] else None
    # end to end: operator from pinned host memory every step, result block back
    e2e = None
    if not args.skip_e2e:
        A_host = torch.empty((n, n), dtype=torch.float32, pin_memory=True)
        A_host.copy_(A)
        blk = torch.empty((256, 256), device=dev, dtype=torch.float64)
        out = torch.empty((256, 256), dtype=torch.float64, pin_memory=True)
        reps = min(args.steps, 3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            A.copy_(A_host, non_blocking=True)
            h2 = step()
            hm.hm_reconstruct_block(h2, 0, 256, 0, 256, blk)
            out.copy_(blk, non_blocking=True)
            torch.cuda.synchronize()
            del h2
        e2e_ms = (time.perf_counter() - t0) * 1e3 / reps
        e2e = {"value": round(e2e_ms / ws, 2), "unit": "ms", "h2d_bytes_per_step": 4 * n * n,
               "d2h_bytes_per_step": 8 * 256 * 256,
               "path": "pinned host operator -> device copy, hm_compress_hbs, hm_reconstruct_block "
                       "of one leaf block -> pinned host"}
        del A_host
    adj = None if args.skip_adjoint else adjoint_bench(hm, torch, dev, max(3, args.steps), 3)
    mfree = None if args.skip_matrix_free else matrix_free_bench(
        hm, torch, dev, max(3, args.steps), n, 2 * n if n == N_HEAD else 0)
    del op
    batched = None if args.skip_batched else batched_bench(hm, torch, dev)
    cpu = None
    if rank == 0 and ws == 1 and not args.skip_cpu:
        cpu = cpu_baseline_line()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "ms", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"HBS-ID compression (Sec. 4.2-4.3) of the FP32 log-kernel matrix, "
                               f"N={n} points on the ellipse (cos t, 0.5 sin t), leaves "
                               f"{LEAF_HEAD}, tol 1e-7, r={R_HEAD}, dense black box",
                   "n": n, "leaf": LEAF_HEAD, "tol": TOL_HEAD, "r": R_HEAD,
                   "precision": "HM_A32: FP32 operator, FP64 samples (exact-accumulation split "
                                "GEMM on the tensor cores), FP64 peeling, bases and ID",
                   "l2": "operator (17.2 GB at N=65536) larger than L2; no flush needed",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "rel_err": {"frobenius": err, "estimate_E": E,
                    "note": "relative Frobenius error of this run's compressed matrix against the "
                            "FP32 operator over all N^2 entries; E: max over 10 unit vectors"},
        "in_order": in_order,
        "mixed": mixed,
        "fp64": fp64,
        "compress": {"t_compress_ms": round(info["t_compress_ms"], 3),
                     "t_blackbox_ms": round(info["t_blackbox_ms"], 3),
                     "blackbox_share": None if bb_share is None else round(bb_share, 3),
                     "ranks": [info["min_rank"], info["max_rank"]], "saturated": info["saturated"],
                     "cols_A": info["cols_A"], "cols_At": info["cols_At"], "bytes": info["bytes"]},
        "roofline": roof,
        "phases": phases,
        "clocks": clk,
        "gpu_launches": int(launches),
        "e2e": e2e,
        "adjoint": adj,
        "matrix_free": mfree,
        "batched": batched,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
