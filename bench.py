"""Benchmark of the H-matrix BEM hot path on one GB300 (or N replicas).

A step is one pass of the whole path over one synthetic problem:
Morton tree + block tree, near-field assembly, batched ACA, load vector,
FP64 GMRES solve and the FP32-factor / FP64-refinement solve.
Workload: bumped icosphere level 7 (327,680 flat triangles, 8 seeded real
spherical harmonics l <= 4, amplitude 0.1), point source p = (3, 0, 0),
C_leaf = 64, eta = 1.5, ACA eps = 1e-7, FP64 master with FP32 copies,
solves to a relative residual of 1e-12 (1e-8 relative solution accuracy).

`value` is seconds per step (lower is better); the JSON line also carries the
per-phase seconds, H-matvec GB/s, the error of the mixed-precision solution
against the FP64 one, the roofline of the dominant kernel and the CPU oracle
timed on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="bumped icosphere level 7, Galerkin single-layer Laplace, P0",
                panels=327680, leaf_size=64, eta=1.5, aca_eps=1e-7, aca_kmax=64, ss_order=8,
                source=[3.0, 0.0, 0.0], solve_rel_tol=1e-12, inner="fp32 factors + fp32 near field",
                inner_tol=1e-4, restart=int(os.environ.get("HM_BENCH_RESTART", "128")), precond=os.environ.get("HM_BENCH_PRECOND", "1") == "1",
                use_graph=os.environ.get("HM_BENCH_GRAPH", "0") == "1")
METRIC = "H-matrix setup s, H-matvec GB/s, solve s at 1e-8 rel. accuracy: mixed vs FP64"
FLOPS_PER_PAIR = 11  # 3 sub + 3 mul + 2 add (|x-y|^2) + rsqrt + multiply-add (weight)
PAIRS_PER_ENTRY = 49


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


CASE = "precision"

# Nominal ALU peaks of GB300 (152 SMs at 2.07 GHz): FP64 2 DFMA / SM / clock,
# FP32 128 FFMA / SM / clock; FMA = 2 flops.
FP64_PEAK_TFLOPS = 152 * 2.07e9 * 2 * 2 / 1e12   # 1.26
FP32_PEAK_TFLOPS = 152 * 2.07e9 * 128 * 2 / 1e12  # 80.5
# FP32 flops of one pair evaluation in the double-float entry (ACA and the
# regular near field; TwoSum 6, TwoProduct 2 with its FMA counted 2, ...): 93 per pair
FF_FLOPS_PER_PAIR = 93

# DRAM traffic per launch from an ncu capture, valid while the kernel's source
# file is unchanged (sha256 of the file at capture time); null otherwise.
TRAFFIC = {
    "row_kernel.f64": {"source": "paper_1806_11558_gb300/csrc/mv_kernels.cuh",
                       "sha256": "317d8d2539db41cb43c4abddd08fe283fb2cbbf21bc763087ebc67cdb6960454",
                       "bytes_per_launch": 15113751808 + 5691392,
                       "profile": "profiles/row_kernel_f64_precision.md"},
}


def _file_sha(rel):
    import hashlib
    with open(os.path.join(ROOT, rel), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def kernel_table(trace, steps):
    """Traced kernels of the timed region, largest device time first."""
    tot = sum(ms for _, ms in trace.values()) or 1.0
    rows = sorted(trace.items(), key=lambda kv: -kv[1][1])
    return {name: {"launches_per_step": c / steps, "ms_per_step": ms / steps, "ms_per_launch": ms / max(c, 1),
                   "share_of_traced": ms / tot} for name, (c, ms) in rows}


def algorithmic_work(mi, ti, dense_leaves, n):
    """Algorithmic work per launch of each traced kernel: (bound, amount, unit)."""
    u = mi["u_entries"]
    w = mi["lr_entries"] - u
    d = mi["dense_entries"]
    rb, re_, cb, ce = dense_leaves.T
    # the near-field kernel evaluates each mirrored pair of leaves once (the
    # ~2% touching positions among them, handed to the touching-pair kernel,
    # are counted too)
    nf_entries = int(((re_ - rb) * (ce - cb))[rb <= cb].sum())
    K = mi["mean_rank"] * ti["n_adm"]  # sum of ranks = length of t
    nl = (ti["n_clusters"] + 1) // 2  # leaf clusters of the binary cluster tree; partials = sum over them of K_w
    return {
        "row_kernel.f64": ("alu", 2.0 * (d + u), "flop"),
        "col_kernel.f64": ("alu", 2.0 * w, "flop"),
        "row_kernel.f32": ("hbm", 4.0 * (d + u) + 4.0 * (n + K) + 8.0 * n, "byte"),
        "col_kernel.f32": ("hbm", 4.0 * w + 4.0 * n + 4.0 * w * nl / n, "byte"),
        "row_kernel.bf16": ("hbm", 4.0 * d + 2.0 * u + 4.0 * (n + K) + 8.0 * n, "byte"),
        "col_kernel.bf16": ("hbm", 2.0 * w + 4.0 * n + 4.0 * w * nl / n, "byte"),
        "nearfield_kernel": ("alu32", float(nf_entries) * PAIRS_PER_ENTRY * FF_FLOPS_PER_PAIR, "flop"),
        "nearfield_kernel.f64": ("alu", float(nf_entries) * PAIRS_PER_ENTRY * FLOPS_PER_PAIR, "flop"),
        "aca_kernel": ("alu32", float(mi["aca_entries"]) * PAIRS_PER_ENTRY * FF_FLOPS_PER_PAIR, "flop"),
    }


PAIR_FLOPS = {"nearfield_kernel": FF_FLOPS_PER_PAIR, "aca_kernel": FF_FLOPS_PER_PAIR,
              "nearfield_kernel.f64": FLOPS_PER_PAIR}


def roofline_entry(name, kt, wk, peaks, peak_src):
    bound, amount, unit = wk
    t = kt["ms_per_launch"] / 1e3
    if bound == "hbm":
        ach, peak, u, src = amount / t / 1e9, peaks["hbm_gbs"], "GB/s", peak_src + " HBM copy bandwidth"
    elif bound == "alu":
        ach, peak, u, src = amount / t / 1e12, FP64_PEAK_TFLOPS, "TFLOP/s", "nominal FP64 (unit counts x clock)"
    else:
        ach, peak, u, src = amount / t / 1e12, FP32_PEAK_TFLOPS, "TFLOP/s", "nominal FP32 (unit counts x clock)"
    tr = TRAFFIC.get(name)
    traffic = None
    if tr is not None and _file_sha(tr["source"]) == tr["sha256"]:
        traffic = tr["bytes_per_launch"]
    out = {"kernel": name, "bound": "alu" if bound.startswith("alu") else bound, "achieved": ach, "peak": peak,
           "unit": u, "frac": ach / peak, "traffic": traffic, "peak_source": src,
           "algorithmic_" + unit + "s_per_launch": amount, "launch_ms": kt["ms_per_launch"],
           "launches_per_step": kt["launches_per_step"]}
    if name in PAIR_FLOPS:
        # entry-evaluation kernels: evaluations of G (one per quadrature-point pair) per second
        out["kernel_evaluations_per_s"] = amount / PAIR_FLOPS[name] / t
    return out


def _inputs():
    import meshgen
    cfg = meshgen.config(CASE)
    return cfg["V"], cfg["T"]


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        # raw samples (the JSON line carries their summary); HM_BENCH_CLOCKS_CSV keeps them
        self.path = os.environ.get("HM_BENCH_CLOCKS_CSV", "/tmp/hm_clocks_%d.csv" % os.getpid())
        self.gpu = gpu_index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x, world):
    """The largest of the ranks' values (the timed region's max over ranks);
    x itself on one rank.  Works on any process-group backend: NCCL reduces
    a device tensor, gloo a host tensor."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def run_ours(args, rank, world):
    import numpy as np
    import torch
    import paper_1806_11558_gb300 as hm
    from paper_1806_11558_gb300 import build as hb

    hb.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    V, T = _inputs()
    n = T.shape[0]
    Vd = torch.from_numpy(V).to(dev)
    Td = torch.from_numpy(T).to(dev)
    src = torch.tensor([WORKLOAD["source"]], dtype=torch.float64, device=dev)
    f = torch.empty((1, n), dtype=torch.float64, device=dev)
    x64 = torch.zeros(n, dtype=torch.float64, device=dev)
    xmx = torch.zeros(n, dtype=torch.float64, device=dev)
    W = WORKLOAD

    def step(Vdev, Tdev, keep=False):
        t = {}
        e = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        e[0].record(stream)
        tree = hm.hm_build_tree(Vdev, Tdev, eta=W["eta"], leaf_size=W["leaf_size"])
        e[1].record(stream)
        A = hm.hm_assemble(tree, aca_eps=W["aca_eps"], aca_kmax=W["aca_kmax"], ss_order=W["ss_order"],
                           factor_dtype=hm.HM_F32, dense_dtype=hm.HM_F32)
        e[2].record(stream)
        hm.hm_load_vector(tree, src, f)
        e[3].record(stream)
        i64 = hm.hm_solve(A, f[0], x64, rel_tol=W["solve_rel_tol"], restart=W["restart"], max_iter=5000,
                          precond=int(W["precond"]), use_graph=int(W["use_graph"]))
        e[4].record(stream)
        imx = hm.hm_solve(A, f[0], xmx, rel_tol=W["solve_rel_tol"], restart=W["restart"], max_iter=5000, refine=1,
                          inner_tol=W["inner_tol"], inner_dtype=hm.HM_F32, max_refine=50,
                          precond=int(W["precond"]), use_graph=int(W["use_graph"]))
        e[5].record(stream)
        torch.cuda.synchronize()
        t["tree_s"] = e[0].elapsed_time(e[1]) / 1e3
        t["assemble_s"] = e[1].elapsed_time(e[2]) / 1e3
        t["load_s"] = e[2].elapsed_time(e[3]) / 1e3
        t["solve_fp64_s"] = e[3].elapsed_time(e[4]) / 1e3
        t["solve_mixed_s"] = e[4].elapsed_time(e[5]) / 1e3
        t["step_s"] = e[0].elapsed_time(e[5]) / 1e3
        t["minfo"] = hm.hm_matrix_get_info(A)
        t["tinfo"] = hm.hm_tree_get_info(tree)
        t["iters_fp64"] = i64.iters
        t["iters_mixed"] = imx.iters
        t["refine_steps"] = imx.refine_steps
        t["resid_fp64"] = i64.rel_resid
        t["resid_mixed"] = imx.rel_resid
        t["kappa_est"] = i64.kappa_est
        if keep:
            return t, tree, A
        hm.hm_free(A)
        hm.hm_free(tree)
        return t

    if args.profile_step:
        r = step(Vd, Td)
        return {"profile_step": args.case, "step_s": r["step_s"], "aca_s": r["minfo"]["s_aca"],
                "aca_small_sum": r["minfo"]["aca_small_sum"],
                "nearfield_s": r["minfo"]["s_nearfield"], "iters_fp64": r["iters_fp64"],
                "iters_mixed": r["iters_mixed"]}, None
    for _ in range(args.warmup):
        step(Vd, Td)
    barrier(world)
    torch.cuda.synchronize()
    clocks = Clocks(dev.index)
    clocks.start()
    hm.hm_trace_enable(True)
    l0 = hm.hm_kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    results = [step(Vd, Td) for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = hm.hm_kernel_launches() - l0
    hm.hm_trace_enable(False)
    trace = hm.hm_trace_read()
    ck = clocks.stop()
    total_s = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, world)
    per_step = total_s / args.steps

    # mixed vs FP64 solution error, matvec GB/s (separate, untimed for `value`)
    last, tree, A = step(Vd, Td, keep=True)
    err_mixed = float(torch.linalg.norm(xmx - x64) / torch.linalg.norm(x64))
    mi, ti = last["minfo"], last["tinfo"]
    xs = torch.randn(n, dtype=torch.float64, device=dev)
    ys = torch.empty_like(xs)
    mv = {}
    for name, prec, esz in (("fp64", hm.HM_F64, 8), ("fp32", hm.HM_F32, 4)):
        for _ in range(3):
            hm.hm_matvec(A, xs, ys, prec=prec)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        reps = 10
        a0.record(stream)
        for _ in range(reps):
            hm.hm_matvec(A, xs, ys, prec=prec)
        a1.record(stream)
        torch.cuda.synchronize()
        sec = a0.elapsed_time(a1) / 1e3 / reps
        byts = (mi["dense_entries"] + mi["lr_entries"]) * esz + n * 8 * 4
        mv[name] = {"s": sec, "gbs": byts / sec / 1e9, "bytes": byts}
    # BF16 factors: one extra assembly and refined solve, reported beside
    A16 = hm.hm_assemble(tree, aca_eps=W["aca_eps"], aca_kmax=W["aca_kmax"], ss_order=W["ss_order"],
                         factor_dtype=hm.HM_BF16, dense_dtype=hm.HM_F32)
    xbf = torch.zeros_like(x64)
    b0 = torch.cuda.Event(enable_timing=True)
    b1 = torch.cuda.Event(enable_timing=True)
    hm.hm_trace_enable(True)
    b0.record(stream)
    ibf = hm.hm_solve(A16, f[0], xbf, rel_tol=W["solve_rel_tol"], restart=W["restart"], max_iter=5000, refine=1,
                      inner_tol=1e-2, inner_dtype=hm.HM_BF16, max_refine=80, raise_on_noconv=False,
                      precond=int(W["precond"]))
    b1.record(stream)
    torch.cuda.synchronize()
    hm.hm_trace_enable(False)
    bf16_kernels = kernel_table(hm.hm_trace_read(), 1)
    bf16 = {"kernels": {k: v for k, v in bf16_kernels.items() if v["share_of_traced"] > 0.01},
            "solve_s": b0.elapsed_time(b1) / 1e3, "err_vs_fp64": float(torch.linalg.norm(xbf - x64) /
                                                                        torch.linalg.norm(x64)),
            "iters": ibf.iters, "refine_steps": ibf.refine_steps, "rel_resid": ibf.rel_resid}
    hm.hm_free(A16)

    # e2e: the same step through the C ABI from pinned host buffers, host<->device copies timed
    Vh = torch.from_numpy(V).pin_memory()
    Th = torch.from_numpy(T).pin_memory()
    xh = torch.empty(n, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 2))
    torch.cuda.synchronize()
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for _ in range(e2e_steps):
        Vd2 = Vh.to(dev, non_blocking=True)
        Td2 = Th.to(dev, non_blocking=True)
        step(Vd2, Td2)
        xh.copy_(xmx, non_blocking=True)
    c1.record(stream)
    torch.cuda.synchronize()
    e2e_s = c0.elapsed_time(c1) / 1e3 / e2e_steps

    # roofline of the dominant kernel: the traced kernel with the largest
    # device time over the timed steps; achieved = its algorithmic work per
    # launch / its mean launch time (CUDA events on its own stream)
    peaks, peak_src = _peaks()
    leaves = hm.hm_tree_get_leaves(tree, True).cpu().numpy().astype("int64")
    kernels = kernel_table(trace, args.steps)
    work = algorithmic_work(mi, ti, leaves, n)
    roofline = None
    for name, kt in kernels.items():
        if name in work:
            roofline = roofline_entry(name, kt, work[name], peaks, peak_src)
            break
    others = {name: roofline_entry(name, kt, work[name], peaks, peak_src)
              for name, kt in kernels.items() if name in work and (roofline is None or name != roofline["kernel"])}
    nf_s = sum(r["minfo"]["s_nearfield"] for r in results) / len(results)
    aca_s = sum(r["minfo"]["s_aca"] for r in results) / len(results)
    hm.hm_free(A)
    hm.hm_free(tree)

    out = {
        "metric": METRIC, "value": per_step, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 (mixed solve: f32 factors, f64 refinement)",
        "data": "synthetic (seeded bumped icosphere, no dataset)",
        "config": dict(WORKLOAD, parallelism="replicas" if world > 1 else "single GPU",
                       l2="inputs larger than L2 (near field %.1f GB, factors %.1f GB)" % (
                           mi["dense_entries"] * 8 / 1e9, mi["lr_entries"] * 8 / 1e9)),
        "setup_s": sum(r["tree_s"] + r["assemble_s"] for r in results) / len(results),
        "tree_s": sum(r["tree_s"] for r in results) / len(results),
        "assemble_s": sum(r["assemble_s"] for r in results) / len(results),
        "nearfield_s": nf_s, "singular_s": sum(r["minfo"]["s_singular"] for r in results) / len(results),
        "aca_s": aca_s, "aca_small_sum": mi["aca_small_sum"],
        "solve_fp64_s": sum(r["solve_fp64_s"] for r in results) / len(results),
        "solve_mixed_s": sum(r["solve_mixed_s"] for r in results) / len(results),
        "iters_fp64": last["iters_fp64"], "iters_mixed": last["iters_mixed"], "refine_steps": last["refine_steps"],
        "resid_fp64": last["resid_fp64"], "resid_mixed": last["resid_mixed"],
        "kappa_est_fp64_solve": last["kappa_est"], "mixed_vs_fp64_rel_err": err_mixed,
        "bf16": bf16, "matvec": mv, "mean_rank": mi["mean_rank"], "max_rank": mi["max_rank"],
        "dense_entries": mi["dense_entries"], "lr_entries": mi["lr_entries"],
        "roofline": roofline, "kernels": kernels, "rooflines_other": others,
        "clocks": ck, "gpu_launches": int(launches),
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(V.nbytes + T.nbytes),
                "d2h_bytes_per_step": int(n * 8)},
    }
    return out, (V, T, last)


def cpu_oracle_step(V, T, budget_s=20.0, iters=None, seed=0):
    """The oracle, as it stands, on a bounded sample of the workload; returns
    the estimated seconds for one full step and what was sampled."""
    import numpy as np
    import oracle
    oracle.build()
    W = WORKLOAD
    t0 = time.perf_counter()
    tr = oracle.Tree(V, T, W["leaf_size"], W["eta"])
    t_tree = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    quad = oracle.Quad(W["ss_order"])
    # near field: a random sample of dense leaves
    nd = len(tr.dense)
    sd = rng.choice(nd, size=min(nd, 60000), replace=False)
    t0 = time.perf_counter()
    blocks = []
    for b in sd:
        rb, re, cb, ce = tr.dense[b]
        blocks.append(oracle.assemble(tr.V, tr.T, tr.perm[rb:re], tr.perm[cb:ce], quad).ravel())
    t_nf = (time.perf_counter() - t0) * nd / len(sd)
    # ACA: a random sample of admissible leaves
    na = len(tr.adm)
    sa = rng.choice(na, size=min(na, 100000), replace=False)
    t0 = time.perf_counter()
    fac = oracle.aca_blocks(tr.V, tr.T, tr.perm, tr.adm[sa], W["aca_eps"], W["aca_kmax"], quad)
    t_aca = (time.perf_counter() - t0) * na / len(sa)
    # H-matvec: the sampled blocks applied, scaled to the whole matrix
    dense_val = np.concatenate(blocks)
    d_off = np.cumsum([0] + [blk.size for blk in blocks])
    parts, uo, wo, o = [], [], [], 0
    for U, Wf in fac:
        uo.append(o); parts.append(U.T.ravel()); o += U.size
        wo.append(o); parts.append(Wf.T.ravel()); o += Wf.size
    uw = np.concatenate(parts) if parts else np.zeros(1)
    rank = np.array([U.shape[1] for U, _ in fac], dtype=np.int32)
    x = rng.standard_normal(tr.n)
    t0 = time.perf_counter()
    reps = 10
    for _ in range(reps):
        oracle.hmatvec_raw(tr.n, tr.dense[sd], d_off[:-1], dense_val, tr.adm[sa], rank, uo, wo, uw, x)
    t_mv_sample = (time.perf_counter() - t0) / reps
    dense_total = int(((tr.dense[:, 1] - tr.dense[:, 0]) * (tr.dense[:, 3] - tr.dense[:, 2])).sum())
    lr_total = uw.size * na / len(sa)
    t_mv = t_mv_sample * (dense_total + lr_total) / max(1, dense_val.size + uw.size)
    n_mv = (iters or 200)
    t_solve = t_mv * n_mv
    total = t_tree + t_nf + t_aca + t_solve
    sample = ("full Morton + block tree (%.1fs); %d of %d dense leaves and %d of %d admissible leaves (ACA), "
              "drawn uniformly with a fixed seed, times scaled by the leaf counts; H-matvec of the sampled "
              "leaves scaled by stored entries x %d matvecs (the GPU's Krylov steps)" % (t_tree, len(sd), nd,
                                                                                           len(sa), na, n_mv))
    return total, sample, dict(tree_s=t_tree, nearfield_s=t_nf, aca_s=t_aca, solve_s=t_solve)


def run_reference(args, rank, world):
    import meshgen  # noqa: F401
    V, T = _inputs()
    cores = os.cpu_count()
    vals = []
    for _ in range(args.warmup):
        cpu_oracle_step(V, T, seed=1)
    t0 = time.perf_counter()
    for k in range(args.steps):
        v, sample, parts = cpu_oracle_step(V, T, seed=2 + k)
        vals.append(v)
    wall = time.perf_counter() - t0
    val = sum(vals) / len(vals)
    return {"impl": "reference", "metric": METRIC, "value": val, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": val * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded bumped icosphere)",
            "config": dict(WORKLOAD), "cpu_baseline": {"value": val, "unit": "s", "cores": cores, "kind": "oracle",
                                                         "sample": sample, "parts": parts, "wall_s": wall},
            "e2e": {"value": val, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _ev(torch):
    return torch.cuda.Event(enable_timing=True)


def run_large(torch, hm):
    """Large workload: icosphere level 8 (1,310,720 panels), leaf 128, eps 1e-6,
    16 point sources; FP64 form (16 FP64 solves in lockstep) against the
    mixed forms (FP32 near field + BF16 factors, then FP32 factors added from
    the FP64 master; inner solves through the 16-right-hand-side tensor-core
    product, FP64 refinement)."""
    import meshgen
    cfg = meshgen.config("large")
    n = cfg["T"].shape[0]
    V, T = torch.from_numpy(cfg["V"]).cuda(), torch.from_numpy(cfg["T"]).cuda()
    e = [_ev(torch) for _ in range(8)]
    hm.hm_trace_enable(True)
    e[0].record()
    tree = hm.hm_build_tree(V, T, eta=cfg["eta"], leaf_size=cfg["leaf_size"])
    A = hm.hm_assemble(tree, aca_eps=cfg["aca_eps"], aca_kmax=64, ss_order=8, factor_dtype=hm.HM_BF16,
                       dense_dtype=hm.HM_F32)
    e[1].record()
    src = torch.from_numpy(np.ascontiguousarray(cfg["sources"])).cuda()
    F = torch.empty((16, n), dtype=torch.float64, device="cuda")
    hm.hm_load_vector(tree, src, F)
    X = torch.randn((16, n), dtype=torch.float64, device="cuda")
    Y = torch.empty_like(X)
    for _ in range(2):
        hm.hm_matvec_block(A, X, Y, prec=hm.HM_BF16)
    e[2].record()
    for _ in range(5):
        hm.hm_matvec_block(A, X, Y, prec=hm.HM_BF16)
    e[3].record()
    opts = dict(rel_tol=1e-12, restart=128, max_iter=5000, precond=1, batched=1)
    Xm = torch.zeros_like(F)
    e[4].record()
    im = hm.hm_solve(A, F, Xm, refine=1, inner_dtype=hm.HM_BF16, inner_tol=1e-2, max_refine=80, **opts)
    e[5].record()
    X64 = torch.zeros_like(F)
    i64 = hm.hm_solve(A, F, X64, **opts)
    e[6].record()
    torch.cuda.synchronize()
    hm.hm_trace_enable(False)
    # the same refinement with FP32 factors (the copy made from the FP64 master)
    hm.hm_matrix_add_copy(A, hm.HM_F32)
    X32 = torch.zeros_like(F)
    e[7].record()
    i32 = hm.hm_solve(A, F, X32, refine=1, inner_dtype=hm.HM_F32, inner_tol=1e-4, max_refine=40, **opts)
    e8 = _ev(torch)
    e8.record()
    torch.cuda.synchronize()
    err32 = float(torch.max(torch.linalg.norm(X32 - X64, dim=1) / torch.linalg.norm(X64, dim=1)))
    mi = hm.hm_matrix_get_info(A)
    mat_bytes = mi["dense_entries"] * 4 + mi["lr_entries"] * 2
    blk_s = e[2].elapsed_time(e[3]) / 5e3
    err = float(torch.max(torch.linalg.norm(Xm - X64, dim=1) / torch.linalg.norm(X64, dim=1)))
    out = {"workload": "large: icosphere level 8, 1,310,720 panels, leaf 128, eta 1.5, ACA eps 1e-6, 16 sources",
           "setup_s": e[0].elapsed_time(e[1]) / 1e3, "nearfield_s": mi["s_nearfield"], "singular_s": mi["s_singular"],
           "aca_s": mi["s_aca"], "mean_rank": mi["mean_rank"],
           "block_matvec_16rhs": {"s": blk_s, "matrix_gb": mat_bytes / 1e9, "gbs": mat_bytes / blk_s / 1e9},
           "solve_mixed_16rhs_s": e[4].elapsed_time(e[5]) / 1e3, "mixed_iters": im.iters,
           "mixed_refine_steps": im.refine_steps, "mixed_rel_resid": im.rel_resid,
           "solve_fp64_16rhs_s": e[5].elapsed_time(e[6]) / 1e3, "fp64_iters": i64.iters,
           "fp64_rel_resid": i64.rel_resid, "mixed_vs_fp64_max_rel_err": err,
           "solve_mixed_fp32_16rhs_s": e[7].elapsed_time(e8) / 1e3, "mixed_fp32_iters": i32.iters,
           "mixed_fp32_refine_steps": i32.refine_steps, "mixed_fp32_rel_resid": i32.rel_resid,
           "mixed_fp32_vs_fp64_max_rel_err": err32,
           "kernels": kernel_table(hm.hm_trace_read(), 1)}
    hm.hm_free(A)
    hm.hm_free(tree)
    return out


def run_batching(torch, hm):
    """Batching workload: 64 stretched icospheres of levels 3..6 (1.79 M panels
    in all), 4 exterior sources each, ACA eps 1e-5, FP32 copies; everything
    in one forest: one launch per phase for all geometries, then 256 GMRES
    (64 geometries x 4 right-hand sides) in lockstep with FP32 inner solves
    through the tensor-core product and FP64 refinement to 1e-6."""
    import meshgen
    cfg = meshgen.config("batching")
    n = cfg["T"].shape[0]
    V, T = torch.from_numpy(cfg["V"]).cuda(), torch.from_numpy(cfg["T"]).cuda()
    e = [_ev(torch) for _ in range(6)]
    hm.hm_trace_enable(True)
    e[0].record()
    tree = hm.hm_build_forest(V, T, cfg["tri_offsets"].tolist(), eta=cfg["eta"], leaf_size=cfg["leaf_size"])
    e[1].record()
    A = hm.hm_assemble(tree, aca_eps=cfg["aca_eps"], aca_kmax=64, ss_order=8, factor_dtype=hm.HM_F32,
                       dense_dtype=hm.HM_F32)
    e[2].record()
    src = torch.from_numpy(np.ascontiguousarray(cfg["sources"])).cuda()
    F = torch.empty((4, n), dtype=torch.float64, device="cuda")
    hm.hm_load_vector_geom(tree, src, F)
    X = torch.zeros_like(F)
    e[3].record()
    opts = dict(rel_tol=1e-6, restart=60, max_iter=5000, precond=1, batched=1, refine=1, inner_dtype=hm.HM_F32,
                inner_tol=1e-4, max_refine=40)
    info = hm.hm_solve(A, F, X, **opts)
    e[4].record()
    torch.cuda.synchronize()
    hm.hm_trace_enable(False)
    # again, with the block-Jacobi inverses and the multi-RHS panels in place:
    # host-driven Arnoldi loop, then the CUDA-graph loop
    warm = {}
    for name, ug in (("solve_warm_s", 0), ("solve_warm_graph_s", 1)):
        Xw = torch.zeros_like(F)
        a, b = _ev(torch), _ev(torch)
        a.record()
        iw = hm.hm_solve(A, F, Xw, use_graph=ug, **opts)
        b.record()
        torch.cuda.synchronize()
        warm[name] = a.elapsed_time(b) / 1e3
        warm[name.replace("_s", "_iters")] = iw.iters
        warm[name.replace("_s", "_same_x")] = bool(torch.equal(Xw, X))
    mi = hm.hm_matrix_get_info(A)
    out = {"workload": "batching: 64 stretched icospheres, levels 3..6, %d panels, 4 sources each, eps 1e-5" % n,
           "tree_s": e[0].elapsed_time(e[1]) / 1e3, "assemble_s": e[1].elapsed_time(e[2]) / 1e3,
           "aca_s": mi["s_aca"], "nearfield_s": mi["s_nearfield"], "solve_s": e[3].elapsed_time(e[4]) / 1e3,
           "systems": 256, "lockstep_iters": info.iters, "refine_steps": info.refine_steps, **warm,
           "max_rel_resid": info.rel_resid, "kernels": kernel_table(hm.hm_trace_read(), 1)}
    hm.hm_free(A)
    hm.hm_free(tree)
    return out


def run_differentiation(torch, hm):
    """Differentiation workload: icosphere level 6, loss = mean squared misfit
    of the potential at 1,024 points (radius 2.5) against a point source at
    (0,0,3); gradients with respect to the Dirichlet data and the 81,920
    per-panel density coefficients through the adjoint solve."""
    import meshgen
    from paper_1806_11558_gb300.autograd import misfit_loss
    cfg = meshgen.config("differentiation")
    n = cfg["T"].shape[0]
    V, T = torch.from_numpy(cfg["V"]).cuda(), torch.from_numpy(cfg["T"]).cuda()
    e = [_ev(torch) for _ in range(5)]
    e[0].record()
    tree = hm.hm_build_tree(V, T, eta=cfg["eta"], leaf_size=cfg["leaf_size"])
    A = hm.hm_assemble(tree, aca_eps=cfg["aca_eps"], aca_kmax=64, ss_order=8)
    e[1].record()
    src = torch.from_numpy(np.ascontiguousarray(cfg["sources"])).cuda()
    f = torch.empty((1, n), dtype=torch.float64, device="cuda")
    hm.hm_load_vector(tree, src, f)
    pts = torch.from_numpy(np.ascontiguousarray(cfg["points"])).cuda()
    p = np.asarray(cfg["target_source"])
    target = torch.from_numpy(1.0 / (4.0 * np.pi * np.linalg.norm(cfg["points"] - p[None, :], axis=1))).cuda()
    opts = dict(rel_tol=1e-13, restart=128, max_iter=5000, precond=1)
    # the pieces on their own (the first solve also builds the block-Jacobi inverses)
    t = {}
    for name, fn in (("solve_first", lambda: hm.hm_solve(A, f[0], torch.zeros_like(f[0]), **opts)),
                     ("solve", lambda: hm.hm_solve(A, f[0], torch.zeros_like(f[0]), **opts)),
                     ("potential", lambda: hm.hm_potential(tree, pts, f[0].contiguous())),
                     ("solve_adjoint_first", lambda: hm.hm_solve(A, f[0], torch.zeros_like(f[0]), trans=1, **opts)),
                     ("solve_adjoint", lambda: hm.hm_solve(A, f[0], torch.zeros_like(f[0]), trans=1, **opts))):
        a, b = _ev(torch), _ev(torch)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        t[name] = {"device_s": a.elapsed_time(b) / 1e3, "wall_s": time.perf_counter() - w0}
    for it in range(2):  # the first pass also loads torch's own elementwise kernels; the second is timed
        fd = f[0].clone().requires_grad_(True)
        cd = torch.ones(n, dtype=torch.float64, device="cuda", requires_grad=True)
        torch.cuda.synchronize()
        hm.hm_trace_enable(it == 1)
        e[2].record()
        L = misfit_loss(A, tree, fd, cd, pts, target, opts)
        e[3].record()
        L.backward()
        e[4].record()
        torch.cuda.synchronize()
    hm.hm_trace_enable(False)
    out = {"workload": "differentiation: icosphere level 6 (81,920 panels), 1,024 evaluation points, FP64",
           "setup_s": e[0].elapsed_time(e[1]) / 1e3, "forward_s": e[2].elapsed_time(e[3]) / 1e3,
           "backward_s": e[3].elapsed_time(e[4]) / 1e3, "loss": float(L.detach()), "pieces": t,
           "kernels": kernel_table(hm.hm_trace_read(), 1)}
    hm.hm_free(A)
    hm.hm_free(tree)
    return out


def run_blockmv(torch, hm, case="bumped6"):
    """Multi-RHS product case (profiling): a bumped icosphere (level 6, or 7
    with case "precision"), leaf 128, BF16 factors, then FP32 factors added
    from the FP64 master; three 16-right-hand-side tensor-core products each."""
    import meshgen
    cfg = meshgen.config(case)
    n = cfg["T"].shape[0]
    V, T = torch.from_numpy(cfg["V"]).cuda(), torch.from_numpy(cfg["T"]).cuda()
    tree = hm.hm_build_tree(V, T, eta=1.5, leaf_size=128)
    A = hm.hm_assemble(tree, aca_eps=1e-6, aca_kmax=64, ss_order=8, factor_dtype=hm.HM_BF16, dense_dtype=hm.HM_F32)
    X = torch.randn((16, n), dtype=torch.float64, device="cuda")
    Y = torch.empty_like(X)
    mi = hm.hm_matrix_get_info(A)
    out = {"workload": "%s (%d panels), leaf 128, 16-RHS product" % (case, n), "n": n}
    for prec, name, fb in ((hm.HM_BF16, "bf16", 2), (hm.HM_F32, "fp32", 4)):
        if prec == hm.HM_F32:
            hm.hm_matrix_add_copy(A, hm.HM_F32)
        a, b = _ev(torch), _ev(torch)
        hm.hm_matvec_block(A, X, Y, prec=prec)
        a.record()
        for _ in range(3):
            hm.hm_matvec_block(A, X, Y, prec=prec)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / 3
        gb = (mi["dense_entries"] * 4 + mi["lr_entries"] * fb) / 1e9
        out[name] = {"ms": ms, "matrix_gb": gb, "gbs": gb / ms * 1e3}
    hm.hm_free(A)
    hm.hm_free(tree)
    return out


def run_workload(name):
    import torch
    import paper_1806_11558_gb300 as hm
    from paper_1806_11558_gb300 import build as hb
    hb.build()
    fn = {"large": run_large, "batching": run_batching, "differentiation": run_differentiation,
          "blockmv": run_blockmv, "blockmv7": lambda t, h: run_blockmv(t, h, "precision")}[name]
    ck = Clocks(torch.cuda.current_device())
    ck.start()
    out = fn(torch, hm)
    out["clocks"] = ck.stop()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--case", default="precision",
                    help="mesh recipe of meshgen.config (default: the precision workload); other cases are "
                         "for profiling and parity runs, not bench lines")
    ap.add_argument("--profile-step", action="store_true",
                    help="run exactly one step (no warm-up, no extras) and print its phase times")
    ap.add_argument("--workload", default=None, choices=["large", "batching", "differentiation", "blockmv", "blockmv7"],
                    help="measure one of the other workloads once and print its numbers (not a bench line)")
    args = ap.parse_args()
    if args.workload:
        print(json.dumps(run_workload(args.workload)))
        return
    global CASE
    CASE = args.case
    if CASE != "precision":
        # other meshes run with their own recipe's tree and ACA parameters
        import meshgen
        cfg = meshgen.config(CASE)
        WORKLOAD.update(workload="%s (profiling / parity case)" % CASE, panels=int(cfg["T"].shape[0]),
                        leaf_size=cfg["leaf_size"], eta=cfg["eta"], aca_eps=cfg["aca_eps"])
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count()))
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args, rank, world)))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    out, extra = run_ours(args, rank, world)
    if args.profile_step:
        if rank == 0:
            print(json.dumps(out))
        return
    V, T, last = extra
    if rank == 0:
        if not args.no_cpu_baseline:
            v, sample, parts = cpu_oracle_step(V, T, iters=last["iters_fp64"] + last["iters_mixed"])
            out["cpu_baseline"] = {"value": v, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
                                   "sample": sample, "parts": parts}
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
