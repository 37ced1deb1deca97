"""Benchmark of the H-matrix BEM hot path on one GB300 (or N replicas).

Headline workload (default, `--case large`): the unit icosphere of level 8,
1,310,720 flat triangles = 1,310,720 piecewise-constant unknowns, C_leaf = 128,
eta = 1.5, ACA eps = 1e-6, 16 seeded exterior point sources (|p| in [2, 4]).
A step is one pass of the whole path: Morton tree + block tree, near field,
batched ACA (with the FP32 copies of near field and factors), the 16 load
vectors, and the mixed-precision solve of the 16 systems -- lockstep GMRES
whose inner solves run on the FP32 copies through the 16-right-hand-side
tensor-core product, FP64 iterative refinement to a relative residual of
1e-12 (1e-8 relative solution accuracy).

Beside it, in the same run and outside the timed steps: the all-FP64 solve
of the same 16 systems on the last step's matrix (timed once, it takes about a
minute), the BF16-factor form, the H-matvec GB/s (one and 16 right-hand
sides), the error of every mixed solution against the FP64 one, the measured
FMA peaks, and the precision workload (bumped icosphere of level 7, 327,680
panels, one source, FP64 solve + FP32-refined solve) as a secondary object.

`value` is seconds per step (lower is better).
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

METRIC = "H-matrix setup s, H-matvec GB/s, solve s at 1e-8 rel. accuracy: mixed vs FP64"

# the two bench workloads (the other meshgen recipes are profiling / parity cases)
LARGE = dict(workload="unit icosphere level 8, Galerkin single-layer Laplace, P0, 16 point sources",
             case="large", panels=1310720, leaf_size=128, eta=1.5, aca_eps=1e-6, aca_kmax=64, ss_order=8,
             nrhs=16, sources="16 seeded exterior point sources, |p| uniform in [2, 4]", solve_rel_tol=1e-12,
             form="mixed: FP32 near field + FP32 factors; lockstep GMRES whose inner solves use the 16-RHS "
                  "tensor-core product; iterative refinement on the FP64 master, its residuals by the 16-RHS "
                  "double-float product",
             inner_tol=1e-4, restart=128, precond=True, batched=True, resid_df=True, factor_tail_bits=0)
PRECISION = dict(workload="bumped icosphere level 7, Galerkin single-layer Laplace, P0",
                 case="precision", panels=327680, leaf_size=64, eta=1.5, aca_eps=1e-7, aca_kmax=64, ss_order=8,
                 nrhs=1, source=[3.0, 0.0, 0.0], solve_rel_tol=1e-12, inner="fp32 factors + fp32 near field",
                 inner_tol=1e-4, restart=128, precond=True, use_graph=False)
FLOPS_PER_PAIR = 11  # 3 sub + 3 mul + 2 add (|x-y|^2) + rsqrt + multiply-add (weight)
PAIRS_PER_ENTRY = 49
MR = 16  # right-hand sides of one tensor-core pass


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# Nominal ALU peaks of GB300 (152 SMs at 2.07 GHz): FP64 2 DFMA / SM / clock,
# FP32 128 FFMA / SM / clock; FMA = 2 flops.  Used only when no measurement
# (hm_measure_fma_peak) is passed in.
FP64_PEAK_TFLOPS = 152 * 2.07e9 * 2 * 2 / 1e12   # 1.26
FP32_PEAK_TFLOPS = 152 * 2.07e9 * 128 * 2 / 1e12  # 80.5
# FP32 flops of one pair evaluation in the double-float entry (ACA and the
# regular near field; TwoSum 6, TwoProduct 2 with its FMA counted 2, ...): 93 per pair
FF_FLOPS_PER_PAIR = 93
# FP32 flops of one term of the double-float product (TwoProduct 1 + 2, TwoSum 6, two cross-term FMAs 4,
# two adds into the compensation 2), FMAs counted 2: 15 flops in 12 instructions, so the instruction mix
# caps these kernels at 15 / 24 = 0.625 of the FMA peak
DF_FLOPS_PER_TERM = 15

# DRAM traffic per launch from an ncu capture, valid while the kernel's source
# file is unchanged (sha256 of the file at capture time); null otherwise.
TRAFFIC = {
    # ncu capture in the level-6 step of the large workload (unit icosphere level 6, leaf 128, 81,920 panels;
    # the row pass writing into the FP32 Krylov block): 1.7621 GB per launch, 1.0384 x its algorithmic
    # bytes (1.6969 GB); scaled to a level-8 launch by the algorithmic bytes (37.79 GB), traffic growing in
    # proportion with the matrix (sha of the file after adding the input gather of the batched product and
    # unrolling the partial sums of split panels, separate kernels: row_mrhs_kernel's code is the captured one)
    "row_mrhs_kernel.f32": {"source": "paper_1806_11558_gb300/csrc/mrhs.cu",
                            "sha256": "4ee0899318fd414d930ad2ed2b4ea5ee980fbe587824bd3c25fc26cfe9488c7b",
                            "bytes_per_launch": 39242683441,
                            "workload": "large",
                            "profile": "profiles/mrhs_kernels_ico6_solve.md"},
    "row_kernel.f64": {"source": "paper_1806_11558_gb300/csrc/mv_kernels.cuh",
                       "sha256": "317d8d2539db41cb43c4abddd08fe283fb2cbbf21bc763087ebc67cdb6960454",
                       "bytes_per_launch": 15113751808 + 5691392,
                       "workload": "precision",
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
    # FP32 factors with BF16 tails: the trailing terms' entries of U (row pass)
    # and W (column pass) are 2-byte, and the column pass runs once per part
    u16 = mi.get("u_tail_entries", 0)
    w16 = mi.get("lr_tail_entries", 0) - u16
    K16 = mi.get("factor_tail_terms", 0)
    nl = (ti["n_clusters"] + 1) // 2  # leaf clusters of the binary cluster tree; partials = sum over them of K_w
    # 16 right-hand sides: X and t rows as BF16 pairs (16 x 2 x 2 B); the timed solve's row pass writes its
    # rows straight into the block of FP32 Krylov vectors (16 x 4 B)
    xr, yr = 4.0 * MR, 4.0 * MR
    return {
        "row_kernel.f64": ("alu", 2.0 * (d + u), "flop"),
        "col_kernel.f64": ("alu", 2.0 * w, "flop"),
        "row_kernel.f32": ("hbm", 4.0 * (d + u) + 4.0 * (n + K) + 8.0 * n, "byte"),
        "col_kernel.f32": ("hbm", 4.0 * w + 4.0 * n + 4.0 * w * nl / n, "byte"),
        "row_kernel.bf16": ("hbm", 4.0 * d + 2.0 * u + 4.0 * (n + K) + 8.0 * n, "byte"),
        "col_kernel.bf16": ("hbm", 2.0 * w + 4.0 * n + 4.0 * w * nl / n, "byte"),
        "row_mrhs_kernel.f32": ("hbm", 4.0 * (d + u - u16) + 2.0 * u16 + xr * (n + K) + yr * n, "byte"),
        "row_mrhs_kernel.bf16": ("hbm", 4.0 * d + 2.0 * u + xr * (n + K) + yr * n, "byte"),
        "col_bcp_kernel.f32": ("hbm", 4.0 * (w - w16) + xr * (n + K - K16), "byte"),
        "col_bcp_kernel.bf16": ("hbm", (2.0 * w16 + xr * (n + K16)) if K16 else (2.0 * w + xr * (n + K)), "byte"),
        "nearfield_kernel": ("alu32", float(nf_entries) * PAIRS_PER_ENTRY * FF_FLOPS_PER_PAIR, "flop"),
        # double-float product of the FP64 master, 16 right-hand sides per launch: DF_FLOPS_PER_TERM per
        # (entry, right-hand side)
        "row_df_kernel": ("alu32", DF_FLOPS_PER_TERM * MR * (d + u), "flop"),
        "col_df_kernel": ("alu32", DF_FLOPS_PER_TERM * MR * w, "flop"),
        "nearfield_kernel.f64": ("alu", float(nf_entries) * PAIRS_PER_ENTRY * FLOPS_PER_PAIR, "flop"),
        "aca_kernel": ("alu32", float(mi["aca_entries"]) * PAIRS_PER_ENTRY * FF_FLOPS_PER_PAIR, "flop"),
    }


PAIR_FLOPS = {"nearfield_kernel": FF_FLOPS_PER_PAIR, "aca_kernel": FF_FLOPS_PER_PAIR,
              "nearfield_kernel.f64": FLOPS_PER_PAIR}


def roofline_entry(name, kt, wk, peaks, peak_src):
    """Roofline object of one traced kernel.  peaks: hbm_gbs (the driver's
    copy bandwidth) and, when measured in this run, fp64_tflops / fp32_tflops
    (hm_measure_fma_peak); the nominal unit-count figures otherwise."""
    bound, amount, unit = wk
    t = kt["ms_per_launch"] / 1e3
    if bound == "hbm":
        ach, peak, u, src = amount / t / 1e9, peaks["hbm_gbs"], "GB/s", peak_src + " HBM copy bandwidth"
    elif bound == "alu":
        ach, u = amount / t / 1e12, "TFLOP/s"
        if "fp64_tflops" in peaks:
            peak, src = peaks["fp64_tflops"], "measured FP64 FMA throughput (hm_measure_fma_peak, this run)"
        else:
            peak, src = FP64_PEAK_TFLOPS, "nominal FP64 (unit counts x clock)"
    else:
        ach, u = amount / t / 1e12, "TFLOP/s"
        if "fp32_tflops" in peaks:
            peak, src = peaks["fp32_tflops"], "measured FP32 FMA throughput (hm_measure_fma_peak, this run)"
        else:
            peak, src = FP32_PEAK_TFLOPS, "nominal FP32 (unit counts x clock)"
    tr = TRAFFIC.get(name)
    traffic = None
    if tr is not None and tr.get("workload") == peaks.get("workload") and _file_sha(tr["source"]) == tr["sha256"]:
        traffic = tr["bytes_per_launch"]
    out = {"kernel": name, "bound": "alu" if bound.startswith("alu") else bound, "achieved": ach, "peak": peak,
           "unit": u, "frac": ach / peak, "traffic": traffic, "peak_source": src,
           "algorithmic_" + unit + "s_per_launch": amount, "launch_ms": kt["ms_per_launch"],
           "launches_per_step": kt["launches_per_step"]}
    if name in PAIR_FLOPS:
        # entry-evaluation kernels: evaluations of G (one per quadrature-point pair) per second
        out["kernel_evaluations_per_s"] = amount / PAIR_FLOPS[name] / t
    return out


def rooflines(trace, steps, mi, ti, leaves, n, peaks, peak_src):
    """(dominant kernel's roofline, the others') from a trace of `steps` steps."""
    kernels = kernel_table(trace, steps)
    work = algorithmic_work(mi, ti, leaves, n)
    dom, others = None, {}
    for name, kt in kernels.items():
        if name not in work:
            continue
        r = roofline_entry(name, kt, work[name], peaks, peak_src)
        if dom is None:
            dom = r
        else:
            others[name] = r
    return dom, others, kernels


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


def _ev(torch):
    return torch.cuda.Event(enable_timing=True)


def _mean(rs, key):
    return sum(r[key] for r in rs) / len(rs)


def measured_fma_peaks(hm, torch):
    """FP64 and FP32 FMA throughput measured now, with the SM clock sampled
    around the measurement."""
    ck = Clocks(torch.cuda.current_device())
    ck.start()
    f64 = hm.hm_measure_fma_peak(hm.HM_F64)
    f32 = hm.hm_measure_fma_peak(hm.HM_F32)
    c = ck.stop()
    return {"fp64_tflops": f64, "fp32_tflops": f32, "sm_mhz": c.get("sm_mhz"),
            "how": "hm_measure_fma_peak: every SM full of threads running 8 independent FMA chains each; best of 3 "
                   "CUDA-event-timed launches"}


# ---------------------------------------------------------------------------
# the headline: level 8, 16 sources, mixed 16-system solve
# ---------------------------------------------------------------------------
def run_large(args, world, hm, torch, W=LARGE, case="large"):
    import meshgen
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    stream = torch.cuda.current_stream()
    cfg = meshgen.config(case)
    V, T = cfg["V"], cfg["T"]
    n = T.shape[0]
    R = W["nrhs"]
    Vd = torch.from_numpy(V).to(dev)
    Td = torch.from_numpy(T).to(dev)
    srcd = torch.from_numpy(np.ascontiguousarray(cfg["sources"][:R])).to(dev)
    F = torch.empty((R, n), dtype=torch.float64, device=dev)
    X = torch.zeros((R, n), dtype=torch.float64, device=dev)
    opts = dict(rel_tol=W["solve_rel_tol"], restart=W["restart"], max_iter=5000, precond=int(W["precond"]),
                batched=1)

    def step(Vdev, Tdev, sdev, keep=False):
        e = [_ev(torch) for _ in range(5)]
        e[0].record(stream)
        tree = hm.hm_build_tree(Vdev, Tdev, eta=W["eta"], leaf_size=W["leaf_size"])
        e[1].record(stream)
        A = hm.hm_assemble(tree, aca_eps=W["aca_eps"], aca_kmax=W["aca_kmax"], ss_order=W["ss_order"],
                           factor_dtype=hm.HM_F32, dense_dtype=hm.HM_F32,
                           factor_tail_bits=W.get("factor_tail_bits", 0))
        e[2].record(stream)
        hm.hm_load_vector(tree, sdev, F)
        e[3].record(stream)
        info = hm.hm_solve(A, F, X, refine=1, inner_dtype=hm.HM_F32, inner_tol=W["inner_tol"], max_refine=40,
                           resid_df=int(W.get("resid_df", False)), **opts)
        e[4].record(stream)
        torch.cuda.synchronize()
        mi = hm.hm_matrix_get_info(A)
        t = {"tree_s": e[0].elapsed_time(e[1]) / 1e3, "assemble_s": e[1].elapsed_time(e[2]) / 1e3,
             "load_s": e[2].elapsed_time(e[3]) / 1e3, "solve_mixed_s": e[3].elapsed_time(e[4]) / 1e3,
             "step_s": e[0].elapsed_time(e[4]) / 1e3, "minfo": mi, "tinfo": hm.hm_tree_get_info(tree),
             "iters": info.iters, "refine_steps": info.refine_steps, "rel_resid": info.rel_resid,
             "inner_dtype": info.inner_dtype}
        if keep:
            return t, tree, A
        hm.hm_free(A)
        hm.hm_free(tree)
        return t

    if args.profile_step:
        r = step(Vd, Td, srcd)
        return {"profile_step": case, "step_s": r["step_s"], "aca_s": r["minfo"]["s_aca"],
                "nearfield_s": r["minfo"]["s_nearfield"], "solve_mixed_s": r["solve_mixed_s"],
                "iters": r["iters"], "refine_steps": r["refine_steps"]}, None
    for _ in range(args.warmup):
        step(Vd, Td, srcd)
    peaks, peak_src = _peaks()
    peaks = dict(peaks, workload=case, **measured_fma_peaks(hm, torch))
    barrier(world)
    torch.cuda.synchronize()
    clocks = Clocks(dev.index)
    clocks.start()
    hm.hm_trace_enable(True)
    l0 = hm.hm_kernel_launches()
    ev0, ev1 = _ev(torch), _ev(torch)
    ev0.record(stream)
    results = [step(Vd, Td, srcd) for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = hm.hm_kernel_launches() - l0
    hm.hm_trace_enable(False)
    trace = hm.hm_trace_read()
    ck = clocks.stop()
    total_s = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, world)
    per_step = total_s / args.steps

    # e2e: the same step through the C ABI from pinned host buffers, host<->device copies timed (right
    # after the timed steps, with the library's block cache as they left it)
    Vh = torch.from_numpy(V).pin_memory()
    Th = torch.from_numpy(T).pin_memory()
    Sh = torch.from_numpy(np.ascontiguousarray(cfg["sources"][:R])).pin_memory()
    Xh = torch.empty((R, n), dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 2))
    torch.cuda.synchronize()
    c0, c1 = _ev(torch), _ev(torch)
    c0.record(stream)
    for _ in range(e2e_steps):
        step(Vh.to(dev, non_blocking=True), Th.to(dev, non_blocking=True), Sh.to(dev, non_blocking=True))
        Xh.copy_(X, non_blocking=True)
    c1.record(stream)
    torch.cuda.synchronize()
    e2e_s = c0.elapsed_time(c1) / 1e3 / e2e_steps

    # --- outside the timed steps: the last step kept, FP64 form, BF16 form, products
    last, tree, A = step(Vd, Td, srcd, keep=True)
    Xm = X.clone()
    mi, ti = last["minfo"], last["tinfo"]
    # the FP64 residual of the mixed solutions (one FP64 product per system)
    HX = torch.empty_like(F)
    hm.hm_matvec(A, Xm, HX, prec=hm.HM_F64)
    resid64 = float(torch.max(torch.linalg.norm(F - HX, dim=1) / torch.linalg.norm(F, dim=1)))
    X64 = torch.zeros_like(F)
    a, b = _ev(torch), _ev(torch)
    a.record(stream)
    i64 = hm.hm_solve(A, F, X64, **opts)
    b.record(stream)
    torch.cuda.synchronize()
    fp64_s = a.elapsed_time(b) / 1e3
    nx64 = torch.linalg.norm(X64, dim=1)
    err32 = float(torch.max(torch.linalg.norm(Xm - X64, dim=1) / nx64))
    # BF16 factors (the copy added from the FP64 master) + FP64 refinement
    hm.hm_matrix_add_copy(A, hm.HM_BF16)
    Xb = torch.zeros_like(F)
    a.record(stream)
    ib = hm.hm_solve(A, F, Xb, refine=1, inner_dtype=hm.HM_BF16, inner_tol=1e-2, max_refine=80,
                     resid_df=int(W.get("resid_df", False)), raise_on_noconv=False, **opts)
    b.record(stream)
    torch.cuda.synchronize()
    bf16_s = a.elapsed_time(b) / 1e3
    errbf = float(torch.max(torch.linalg.norm(Xb - X64, dim=1) / nx64))
    # H-matvec: 16 right-hand sides on the tensor cores, one right-hand side on the CUDA cores
    Xr = torch.randn((R, n), dtype=torch.float64, device=dev)
    Yr = torch.empty_like(Xr)
    mv = {}
    for name, prec, fb in (("16rhs_fp32", hm.HM_F32, 4), ("16rhs_bf16", hm.HM_BF16, 2)):
        hm.hm_matvec_block(A, Xr, Yr, prec=prec)
        a.record(stream)
        for _ in range(5):
            hm.hm_matvec_block(A, Xr, Yr, prec=prec)
        b.record(stream)
        torch.cuda.synchronize()
        sec = a.elapsed_time(b) / 5e3
        byts = mi["dense_entries"] * 4 + mi["lr_entries"] * fb
        mv[name] = {"s": sec, "matrix_gb": byts / 1e9, "gbs_matrix": byts / sec / 1e9,
                    "s_per_rhs": sec / R}
    # the FP64 master, 16 right-hand sides in double-float arithmetic (the residual product of the refinement)
    hm.hm_matvec_block(A, Xr, Yr, prec=hm.HM_F64)
    a.record(stream)
    for _ in range(3):
        hm.hm_matvec_block(A, Xr, Yr, prec=hm.HM_F64)
    b.record(stream)
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 3e3
    byts = (mi["dense_entries"] + mi["lr_entries"]) * 8
    mv["16rhs_df64"] = {"s": sec, "matrix_gb": byts / 1e9, "gbs_matrix": byts / sec / 1e9, "s_per_rhs": sec / R}
    for name, prec, esz in (("1rhs_fp64", hm.HM_F64, 8), ("1rhs_fp32", hm.HM_F32, 4)):
        hm.hm_matvec(A, Xr[0], Yr[0], prec=prec)
        a.record(stream)
        for _ in range(3):
            hm.hm_matvec(A, Xr[0], Yr[0], prec=prec)
        b.record(stream)
        torch.cuda.synchronize()
        sec = a.elapsed_time(b) / 3e3
        byts = (mi["dense_entries"] + mi["lr_entries"]) * esz + n * 8 * 4
        mv[name] = {"s": sec, "gbs": byts / sec / 1e9, "bytes": byts}
    leaves = hm.hm_tree_get_leaves(tree, True).cpu().numpy().astype("int64")
    dom, others, kernels = rooflines(trace, args.steps, mi, ti, leaves, n, peaks, peak_src)
    hm.hm_free(A)
    hm.hm_free(tree)


    out = {
        "metric": METRIC, "value": per_step, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 (mixed solve: f32 near field + f32 factors, f64 refinement)",
        "data": "synthetic (seeded unit icosphere and point sources, no dataset)",
        "config": dict(W, parallelism="replicas" if world > 1 else "single GPU",
                       l2="inputs larger than L2 (near field %.1f GB, factors %.1f GB in FP64)" % (
                           mi["dense_entries"] * 8 / 1e9, mi["lr_entries"] * 8 / 1e9)),
        "setup_s": _mean(results, "tree_s") + _mean(results, "assemble_s"),
        "tree_s": _mean(results, "tree_s"), "assemble_s": _mean(results, "assemble_s"),
        "nearfield_s": sum(r["minfo"]["s_nearfield"] for r in results) / len(results),
        "singular_s": sum(r["minfo"]["s_singular"] for r in results) / len(results),
        "aca_s": sum(r["minfo"]["s_aca"] for r in results) / len(results),
        "load_s": _mean(results, "load_s"),
        "solve_mixed_16rhs_s": _mean(results, "solve_mixed_s"),
        "mixed_iters": last["iters"], "mixed_refine_steps": last["refine_steps"],
        "mixed_rel_resid": last["rel_resid"], "mixed_inner_dtype": last["inner_dtype"],
        "mixed_rel_resid_fp64": resid64,
        "fp64_16rhs": {"solve_s": fp64_s, "repetitions": 1, "iters": i64.iters, "rel_resid": i64.rel_resid,
                       "note": "the all-FP64 GPU form of the same 16 systems (lockstep GMRES, FP64 products), "
                               "timed once on the last step's matrix"},
        "mixed_vs_fp64_rel_err": err32,
        "mixed_vs_fp64_time_ratio": fp64_s / _mean(results, "solve_mixed_s"),
        "bf16_16rhs": {"solve_s": bf16_s, "repetitions": 1, "iters": ib.iters, "refine_steps": ib.refine_steps,
                       "rel_resid": ib.rel_resid, "inner_dtype": ib.inner_dtype, "err_vs_fp64": errbf,
                       "note": "BF16 factors added from the FP64 master, FP32 near field, inner tol 1e-2, "
                               "residuals as the headline's"},
        "matvec": mv, "mean_rank": mi["mean_rank"], "max_rank": mi["max_rank"],
        "dense_entries": mi["dense_entries"], "lr_entries": mi["lr_entries"],
        "aca_tuned": {"small_sum": mi["aca_small_sum"], "threads": mi["aca_threads"],
                      "ctas_per_sm": mi["aca_ctas_per_sm"]},
        "roofline": dom, "rooflines_other": others, "kernels": kernels,
        "measured_peaks": {k: peaks[k] for k in ("fp64_tflops", "fp32_tflops", "sm_mhz", "how")},
        "clocks": ck, "gpu_launches": int(launches),
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(V.nbytes + T.nbytes + Sh.numel() * 8),
                "d2h_bytes_per_step": int(R * n * 8)},
    }
    return out, (V, T, {"iters_fp64": i64.iters, "n_systems": R, "W": W, "case": case,
                        "fma_peaks": out["measured_peaks"]})


# ---------------------------------------------------------------------------
# the precision workload (one source): FP64 solve + FP32-refined solve
# ---------------------------------------------------------------------------
def run_single(args, world, hm, torch, W=PRECISION, case="precision", extras=True, fma_peaks=None):
    import meshgen
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    stream = torch.cuda.current_stream()
    cfg = meshgen.config(case)
    V, T = cfg["V"], cfg["T"]
    n = T.shape[0]
    Vd = torch.from_numpy(V).to(dev)
    Td = torch.from_numpy(T).to(dev)
    src = torch.tensor([W["source"]], dtype=torch.float64, device=dev)
    f = torch.empty((1, n), dtype=torch.float64, device=dev)
    x64 = torch.zeros(n, dtype=torch.float64, device=dev)
    xmx = torch.zeros(n, dtype=torch.float64, device=dev)
    sopts = dict(rel_tol=W["solve_rel_tol"], restart=W["restart"], max_iter=5000, precond=int(W["precond"]),
                 use_graph=int(W["use_graph"]))

    def step(Vdev, Tdev, keep=False):
        e = [_ev(torch) for _ in range(6)]
        e[0].record(stream)
        tree = hm.hm_build_tree(Vdev, Tdev, eta=W["eta"], leaf_size=W["leaf_size"])
        e[1].record(stream)
        A = hm.hm_assemble(tree, aca_eps=W["aca_eps"], aca_kmax=W["aca_kmax"], ss_order=W["ss_order"],
                           factor_dtype=hm.HM_F32, dense_dtype=hm.HM_F32)
        e[2].record(stream)
        hm.hm_load_vector(tree, src, f)
        e[3].record(stream)
        i64 = hm.hm_solve(A, f[0], x64, **sopts)
        e[4].record(stream)
        imx = hm.hm_solve(A, f[0], xmx, refine=1, inner_tol=W["inner_tol"], inner_dtype=hm.HM_F32, max_refine=50,
                          **sopts)
        e[5].record(stream)
        torch.cuda.synchronize()
        t = {"tree_s": e[0].elapsed_time(e[1]) / 1e3, "assemble_s": e[1].elapsed_time(e[2]) / 1e3,
             "load_s": e[2].elapsed_time(e[3]) / 1e3, "solve_fp64_s": e[3].elapsed_time(e[4]) / 1e3,
             "solve_mixed_s": e[4].elapsed_time(e[5]) / 1e3, "step_s": e[0].elapsed_time(e[5]) / 1e3,
             "minfo": hm.hm_matrix_get_info(A), "tinfo": hm.hm_tree_get_info(tree), "iters_fp64": i64.iters,
             "iters_mixed": imx.iters, "refine_steps": imx.refine_steps, "resid_fp64": i64.rel_resid,
             "resid_mixed": imx.rel_resid, "kappa_est": i64.kappa_est}
        if keep:
            return t, tree, A
        hm.hm_free(A)
        hm.hm_free(tree)
        return t

    if args.profile_step and extras:
        r = step(Vd, Td)
        return {"profile_step": case, "step_s": r["step_s"], "aca_s": r["minfo"]["s_aca"],
                "aca_small_sum": r["minfo"]["aca_small_sum"], "nearfield_s": r["minfo"]["s_nearfield"],
                "iters_fp64": r["iters_fp64"], "iters_mixed": r["iters_mixed"]}, None
    warmup = args.warmup if extras else 1
    steps = args.steps if extras else 2
    for _ in range(warmup):
        step(Vd, Td)
    peaks, peak_src = _peaks()
    peaks = dict(peaks, workload=case, **(fma_peaks or measured_fma_peaks(hm, torch)))
    barrier(world)
    torch.cuda.synchronize()
    clocks = Clocks(dev.index)
    clocks.start()
    hm.hm_trace_enable(True)
    l0 = hm.hm_kernel_launches()
    ev0, ev1 = _ev(torch), _ev(torch)
    ev0.record(stream)
    results = [step(Vd, Td) for _ in range(steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = hm.hm_kernel_launches() - l0
    hm.hm_trace_enable(False)
    trace = hm.hm_trace_read()
    ck = clocks.stop()
    per_step = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, world) / steps
    last, tree, A = step(Vd, Td, keep=True)
    err_mixed = float(torch.linalg.norm(xmx - x64) / torch.linalg.norm(x64))
    mi, ti = last["minfo"], last["tinfo"]
    summary = {
        "value": per_step, "unit": "s", "steps": steps, "warmup": warmup,
        "config": dict(W, l2="inputs larger than L2 (near field %.1f GB, factors %.1f GB)" % (
            mi["dense_entries"] * 8 / 1e9, mi["lr_entries"] * 8 / 1e9)),
        "setup_s": _mean(results, "tree_s") + _mean(results, "assemble_s"),
        "tree_s": _mean(results, "tree_s"), "assemble_s": _mean(results, "assemble_s"),
        "nearfield_s": sum(r["minfo"]["s_nearfield"] for r in results) / len(results),
        "singular_s": sum(r["minfo"]["s_singular"] for r in results) / len(results),
        "aca_s": sum(r["minfo"]["s_aca"] for r in results) / len(results),
        "solve_fp64_s": _mean(results, "solve_fp64_s"), "solve_mixed_s": _mean(results, "solve_mixed_s"),
        "iters_fp64": last["iters_fp64"], "iters_mixed": last["iters_mixed"], "refine_steps": last["refine_steps"],
        "resid_fp64": last["resid_fp64"], "resid_mixed": last["resid_mixed"],
        "kappa_est_fp64_solve": last["kappa_est"], "mixed_vs_fp64_rel_err": err_mixed,
        "mean_rank": mi["mean_rank"], "max_rank": mi["max_rank"], "dense_entries": mi["dense_entries"],
        "lr_entries": mi["lr_entries"], "clocks": ck, "gpu_launches": int(launches),
    }
    leaves = hm.hm_tree_get_leaves(tree, True).cpu().numpy().astype("int64")
    dom, others, kernels = rooflines(trace, steps, mi, ti, leaves, n, peaks, peak_src)
    summary["roofline"] = dom
    summary["rooflines_other"] = others
    if not extras:
        summary["kernels"] = {k: v for k, v in kernels.items() if v["share_of_traced"] > 0.02}
        hm.hm_free(A)
        hm.hm_free(tree)
        return summary
    xs = torch.randn(n, dtype=torch.float64, device=dev)
    ys = torch.empty_like(xs)
    mv = {}
    for name, prec, esz in (("fp64", hm.HM_F64, 8), ("fp32", hm.HM_F32, 4)):
        for _ in range(3):
            hm.hm_matvec(A, xs, ys, prec=prec)
        a, b = _ev(torch), _ev(torch)
        a.record(stream)
        for _ in range(10):
            hm.hm_matvec(A, xs, ys, prec=prec)
        b.record(stream)
        torch.cuda.synchronize()
        sec = a.elapsed_time(b) / 1e4
        byts = (mi["dense_entries"] + mi["lr_entries"]) * esz + n * 8 * 4
        mv[name] = {"s": sec, "gbs": byts / sec / 1e9, "bytes": byts}
    hm.hm_free(A)
    hm.hm_free(tree)
    Vh = torch.from_numpy(V).pin_memory()
    Th = torch.from_numpy(T).pin_memory()
    xh = torch.empty(n, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(steps, 2))
    torch.cuda.synchronize()
    c0, c1 = _ev(torch), _ev(torch)
    c0.record(stream)
    for _ in range(e2e_steps):
        step(Vh.to(dev, non_blocking=True), Th.to(dev, non_blocking=True))
        xh.copy_(xmx, non_blocking=True)
    c1.record(stream)
    torch.cuda.synchronize()
    e2e_s = c0.elapsed_time(c1) / 1e3 / e2e_steps
    out = {"metric": METRIC, "n_gpus": world, "ms_per_step": per_step * 1e3, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64 (mixed solve: f32 factors, f64 refinement)",
           "data": "synthetic (seeded bumped icosphere, no dataset)", **summary,
           "config": dict(summary["config"], parallelism="replicas" if world > 1 else "single GPU"),
           "matvec": mv, "kernels": kernels,
           "measured_peaks": {k: peaks[k] for k in ("fp64_tflops", "fp32_tflops", "sm_mhz", "how")},
           "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(V.nbytes + T.nbytes),
                   "d2h_bytes_per_step": int(n * 8)}}
    return out, (V, T, {"iters_fp64": last["iters_fp64"], "n_systems": 1, "W": W, "case": case,
                        "fma_peaks": out["measured_peaks"]})


# ---------------------------------------------------------------------------
# the CPU oracle on a bounded sample of the workload
# ---------------------------------------------------------------------------
# Admissible leaves drawn per size class (rows = columns; 80 .. 81,920 at level
# 8 with leaf 128, 40 .. 40,960 at level 7 with leaf 64): many of the small
# ones, at least one of the largest.
ACA_SAMPLE = {40: 6000, 80: 4000, 160: 2000, 320: 1000, 640: 400, 1280: 160, 2560: 48, 5120: 16, 10240: 8,
              20480: 4, 40960: 2, 81920: 1}
# Lockstep Arnoldi steps of the all-FP64 GPU solve of each workload (block-
# Jacobi preconditioned), the iteration count of the CPU estimate's solve
# when the GPU arm has not run in the same process.
FP64_STEPS = {"large": 111, "precision": 84}


class OracleTree:
    """The oracle's tree of a workload, built once per process and timed."""
    cache = {}

    @classmethod
    def get(cls, case, V, T, leaf, eta):
        import oracle
        if case not in cls.cache:
            oracle.build()
            t0 = time.perf_counter()
            tr = oracle.Tree(V, T, leaf, eta)
            cls.cache[case] = (tr, time.perf_counter() - t0)
        return cls.cache[case]


def cpu_oracle_step(case, V, T, W, n_systems, iters_per_system, seed=0, dense_sample=2000, gmres_steps=3):
    """The oracle, as it stands, on a bounded sample of one step of the
    workload.  Returns (estimated seconds of a full step, measured seconds of
    the sampled work, description, parts).

    What runs: the oracle's tree of the whole mesh (built once per process and
    timed then); the near field of `dense_sample` dense leaves drawn uniformly;
    the ACA of admissible leaves drawn per size class (ACA_SAMPLE); and
    oracle.gmres on the sampled operator (those leaves only, at the full
    dimension n) for `gmres_steps` Arnoldi steps, its products timed apart
    from its orthogonalisation.  The estimate scales each sampled part to the
    whole workload: near field by the leaf count, each ACA size class by its
    leaf count and by the thread parallelism the class had in the sample, the
    solve by n_systems x iters_per_system Arnoldi steps of a product scaled
    to the stored entries of the whole matrix plus the measured
    orthogonalisation cost per step (at the sampled depth)."""
    import oracle
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    tr, t_tree = OracleTree.get(case, V, T, W["leaf_size"], W["eta"])
    rng = np.random.default_rng(seed)
    quad = oracle.Quad(W["ss_order"])
    w0 = time.perf_counter()
    nd = len(tr.dense)
    sd = np.sort(rng.choice(nd, size=min(nd, dense_sample), replace=False))
    t0 = time.perf_counter()
    blocks = []
    for b in sd:
        rb, re, cb, ce = tr.dense[b]
        blocks.append(oracle.assemble(tr.V, tr.T, tr.perm[rb:re], tr.perm[cb:ce], quad).ravel())
    t_nf = (time.perf_counter() - t0) * nd / len(sd)
    sizes = tr.adm[:, 1] - tr.adm[:, 0]
    t_aca, fac, sa_all, aca_note = 0.0, [], [], []
    for sz in np.unique(sizes):
        idx = np.flatnonzero(sizes == sz)
        k = min(len(idx), ACA_SAMPLE.get(int(sz), 16))
        sa = np.sort(rng.choice(idx, size=k, replace=False))
        t0 = time.perf_counter()
        fac += oracle.aca_blocks(tr.V, tr.T, tr.perm, tr.adm[sa], W["aca_eps"], W["aca_kmax"], quad)
        dt = time.perf_counter() - t0
        # the class's blocks run on min(count, cores) threads in a full run,
        # on min(k, cores) in the sample
        t_aca += dt * (len(idx) / k) * (min(k, cores) / min(len(idx), cores))
        sa_all.append(sa)
        aca_note.append("%d/%d" % (k, len(idx)))
    sa_all = np.concatenate(sa_all)
    # the sampled operator, applied by oracle.gmres
    dense_val = np.concatenate(blocks)
    d_off = np.cumsum([0] + [blk.size for blk in blocks])[:-1]
    parts, uo, wo, o = [], [], [], 0
    for U, Wf in fac:
        uo.append(o)
        parts.append(U.T.ravel())
        o += U.size
        wo.append(o)
        parts.append(Wf.T.ravel())
        o += Wf.size
    uw = np.concatenate(parts) if parts else np.zeros(1)
    rank = np.array([U.shape[1] for U, _ in fac], dtype=np.int32)
    t_mv = [0.0, 0]

    def mv_sample(xm):
        t1 = time.perf_counter()
        y = oracle.hmatvec_raw(tr.n, tr.dense[sd], d_off, dense_val, tr.adm[sa_all], rank, uo, wo, uw, xm)
        t_mv[0] += time.perf_counter() - t1
        t_mv[1] += 1
        return y

    b = rng.standard_normal(tr.n)
    t0 = time.perf_counter()
    oracle.gmres(mv_sample, b, restart=30, tol=1e-300, maxiter=gmres_steps)
    t_gm = time.perf_counter() - t0
    wall = time.perf_counter() - w0
    dense_total = int(((tr.dense[:, 1] - tr.dense[:, 0]) * (tr.dense[:, 3] - tr.dense[:, 2])).sum())
    # stored factor entries of the whole matrix: the sampled mean per leaf of each size class
    lr_total = 0.0
    for sz in np.unique(sizes):
        pick = sizes[sa_all] == sz
        ent = np.array([U.size + Wf.size for (U, Wf), p in zip(fac, pick) if p], dtype=np.float64)
        lr_total += ent.mean() * np.count_nonzero(sizes == sz) if ent.size else 0.0
    scale = (dense_total + lr_total) / max(1, dense_val.size + uw.size)
    per_mv = t_mv[0] / max(1, t_mv[1])
    per_step_other = max(0.0, t_gm - t_mv[0]) / gmres_steps
    t_solve = n_systems * iters_per_system * (per_mv * scale + per_step_other)
    total = t_tree + t_nf + t_aca + t_solve
    sample = ("oracle tree of the whole mesh (%.1f s, built once per process); near field of %d of %d dense "
              "leaves (uniform draw); ACA of admissible leaves per size class (%s, sampled/total); oracle.gmres on "
              "the sampled operator for %d Arnoldi steps at n = %d. Estimate = tree + near field x %d/%d + ACA per "
              "class x count (thread parallelism corrected) + %d systems x %d Arnoldi steps x (sampled product "
              "x %.0f stored-entry ratio + orthogonalisation per step)"
              % (t_tree, len(sd), nd, ", ".join(aca_note), gmres_steps, tr.n, nd, len(sd), n_systems,
                 iters_per_system, scale))
    return total, wall, sample, dict(tree_s=t_tree, nearfield_s=t_nf, aca_s=t_aca, solve_s=t_solve,
                                     sample_wall_s=wall)


def run_reference(args, rank, world):
    """The reference arm: the oracle on the host cores.  Each step is one
    bounded-sample estimate of a full step (cpu_oracle_step, a fresh sample
    per step); `value` is the mean estimate (marked as such), `ms_per_step` the
    wall time the sampled work of a step actually took."""
    import meshgen
    case = args.case
    W = LARGE if case == "large" else PRECISION
    cfg = meshgen.config(case)
    V, T = cfg["V"], cfg["T"]
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    nsys = W["nrhs"]
    its = FP64_STEPS.get(case, 100)
    t0 = time.perf_counter()
    OracleTree.get(case, V, T, W["leaf_size"], W["eta"])
    t_setup = time.perf_counter() - t0
    for k in range(args.warmup):
        cpu_oracle_step(case, V, T, W, nsys, its, seed=1000 + k)
    vals, walls = [], []
    for k in range(args.steps):
        v, wall, sample, parts = cpu_oracle_step(case, V, T, W, nsys, its, seed=2 + k)
        vals.append(v)
        walls.append(wall)
    val = sum(vals) / len(vals)
    ms = 1e3 * sum(walls) / len(walls)
    return {"impl": "reference", "metric": METRIC, "value": val, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded meshes and sources, no dataset)",
            "value_is_estimate": True,
            "value_note": "each step is one bounded-sample estimate of a full oracle step of this workload "
                          "(see cpu_baseline.sample); value = mean estimate in seconds per full step, "
                          "ms_per_step = wall time of the sampled work one step actually ran",
            "config": dict(W), "cpu_baseline": {"value": val, "unit": "s", "cores": cores, "kind": "oracle",
                                                 "sample": sample, "parts": parts,
                                                 "tree_build_once_s": t_setup,
                                                 "estimates_min_max": [min(vals), max(vals)]},
            "e2e": {"value": val, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_workload(name):
    import torch
    import paper_1806_11558_gb300 as hm
    from paper_1806_11558_gb300 import build as hb
    hb.build()
    fn = {"batching": run_batching, "differentiation": run_differentiation,
          "blockmv": run_blockmv, "blockmv7": lambda t, h: run_blockmv(t, h, "precision"),
          "blockmv_tc": lambda t, h: run_blockmv(t, h, tcgen05=1),
          "blockmv8": lambda t, h: run_blockmv(t, h, "large"),
          "blockmv8_tc": lambda t, h: run_blockmv(t, h, "large", tcgen05=1),
          "blockmv8_tail": lambda t, h: run_blockmv(t, h, "large", tail_bits=12),
          "blockmv_tail": lambda t, h: run_blockmv(t, h, tail_bits=12),
          "solve6": run_solve16,
          "dfmv8": lambda t, h: run_dfmv(t, h, "large"), "dfmv6": lambda t, h: run_dfmv(t, h, "bumped6")}[name]
    ck = Clocks(torch.cuda.current_device())
    ck.start()
    out = fn(torch, hm)
    out["clocks"] = ck.stop()
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
           "max_rel_resid": info.rel_resid,
           "aca_tuned": {"small_sum": mi["aca_small_sum"], "threads": mi["aca_threads"],
                         "ctas_per_sm": mi["aca_ctas_per_sm"]},
           "kernels": kernel_table(hm.hm_trace_read(), 1)}
    hm.hm_free(A)
    hm.hm_free(tree)
    return out


def run_differentiation(torch, hm):
    """Differentiation workload: icosphere level 6, loss = mean squared misfit
    of the potential at 1,024 points (radius 2.5) against a point source at
    (0,0,3); gradients with respect to the Dirichlet data and the 81,920
    per-panel density coefficients through the adjoint solve."""
    import meshgen
    from paper_1806_11558_gb300.autograd import DensitySolve, Potential

    def misfit_loss(A, tree, f, c, points, target, opts):
        # the workload's objective: mean squared misfit of the potential at the points
        alpha = DensitySolve.apply(A, f, c, opts)
        return torch.mean((Potential.apply(tree, points, alpha) - target) ** 2)

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


def run_blockmv(torch, hm, case="bumped6", tcgen05=0, tail_bits=0):
    """Multi-RHS product case (profiling): a bumped icosphere (level 6, or 7
    with case "precision"), leaf 128, BF16 factors, then FP32 factors added
    from the FP64 master (with tail_bits > 0: each block's trailing ACA terms
    in BF16); three 16-right-hand-side tensor-core products each (row pass on
    mma.sync, or on tcgen05 / TMEM with tcgen05 = 1)."""
    import meshgen
    cfg = meshgen.config(case)
    n = cfg["T"].shape[0]
    V, T = torch.from_numpy(cfg["V"]).cuda(), torch.from_numpy(cfg["T"]).cuda()
    tree = hm.hm_build_tree(V, T, eta=1.5, leaf_size=128)
    A = hm.hm_assemble(tree, aca_eps=1e-6, aca_kmax=64, ss_order=8, factor_dtype=hm.HM_BF16, dense_dtype=hm.HM_F32,
                       mrhs_tcgen05=tcgen05, factor_tail_bits=tail_bits)
    X = torch.randn((16, n), dtype=torch.float64, device="cuda")
    Y = torch.empty_like(X)
    mi = hm.hm_matrix_get_info(A)
    ti = hm.hm_tree_get_info(tree)
    out = {"workload": "%s (%d panels), leaf 128, 16-RHS product, row pass on %s%s" % (
               case, n, "tcgen05" if tcgen05 else "mma.sync",
               ", FP32 factors with BF16 tails (2^-%d)" % tail_bits if tail_bits else ""), "n": n,
           "dense_entries": mi["dense_entries"], "u_entries": mi["u_entries"], "lr_entries": mi["lr_entries"],
           "total_rank": mi["mean_rank"] * ti["n_adm"], "factor_tail_terms": mi["factor_tail_terms"],
           "lr_tail_entries": mi["lr_tail_entries"], "u_tail_entries": mi["u_tail_entries"]}
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
        tails = mi["lr_tail_entries"] if prec == hm.HM_F32 else 0
        gb = (mi["dense_entries"] * 4 + (mi["lr_entries"] - tails) * fb + tails * 2) / 1e9
        out[name] = {"ms": ms, "matrix_gb": gb, "gbs": gb / ms * 1e3}
    hm.hm_free(A)
    hm.hm_free(tree)
    return out


def run_solve16(torch, hm, level=6):
    """The large workload's step at a smaller size (profiling): unit icosphere
    of the given level, leaf 128, ACA eps 1e-6, the large workload's 16
    sources, FP32 copies, and its batched refined solve (the same solver
    parameters); one untimed step, then one timed."""
    import meshgen
    W = LARGE
    V, T = meshgen.icosphere(level)
    n = T.shape[0]
    Vd, Td = torch.from_numpy(V).cuda(), torch.from_numpy(T).cuda()
    src = torch.from_numpy(np.ascontiguousarray(meshgen.point_sources(meshgen.MASTER_SEED + 5, W["nrhs"]))).cuda()
    F = torch.empty((W["nrhs"], n), dtype=torch.float64, device="cuda")
    out = {"workload": "unit icosphere level %d (%d panels), leaf 128, 16 sources, the large workload's step" % (
        level, n)}
    for rep in range(2):
        a, b = _ev(torch), _ev(torch)
        a.record()
        tree = hm.hm_build_tree(Vd, Td, eta=W["eta"], leaf_size=W["leaf_size"])
        A = hm.hm_assemble(tree, aca_eps=W["aca_eps"], aca_kmax=W["aca_kmax"], ss_order=W["ss_order"],
                           factor_dtype=hm.HM_F32, dense_dtype=hm.HM_F32)
        hm.hm_load_vector(tree, src, F)
        X = torch.zeros_like(F)
        info = hm.hm_solve(A, F, X, refine=1, inner_dtype=hm.HM_F32, inner_tol=W["inner_tol"], max_refine=40,
                           resid_df=1, rel_tol=W["solve_rel_tol"], restart=W["restart"], max_iter=5000,
                           precond=int(W["precond"]), batched=1)
        b.record()
        torch.cuda.synchronize()
        mi, ti = hm.hm_matrix_get_info(A), hm.hm_tree_get_info(tree)
        out.update(step_s=a.elapsed_time(b) / 1e3, iters=info.iters, refine_steps=info.refine_steps,
                   rel_resid=info.rel_resid, dense_entries=mi["dense_entries"], u_entries=mi["u_entries"],
                   lr_entries=mi["lr_entries"], total_rank=round(mi["mean_rank"] * ti["n_adm"]),
                   row_mrhs_bytes=algorithmic_work(mi, ti, hm.hm_tree_get_leaves(tree, True).cpu().numpy()
                                                   .astype(np.int64), n)["row_mrhs_kernel.f32"][1])
        hm.hm_free(A)
        hm.hm_free(tree)
    return out


def run_dfmv(torch, hm, case):
    """The FP64 master applied to 16 right-hand sides: the double-float
    16-column product (hm_matvec_block, HM_F64) against 16 FP64 products
    (hm_matvec, one right-hand side each), and their difference."""
    import meshgen
    cfg = meshgen.config(case)
    n = cfg["T"].shape[0]
    leaf, eps = (128, 1e-6) if case == "large" else (64, 1e-7)
    V, T = torch.from_numpy(cfg["V"]).cuda(), torch.from_numpy(cfg["T"]).cuda()
    tree = hm.hm_build_tree(V, T, eta=1.5, leaf_size=leaf)
    A = hm.hm_assemble(tree, aca_eps=eps, aca_kmax=64, ss_order=8, factor_dtype=hm.HM_F64, dense_dtype=hm.HM_F64)
    gen = torch.Generator(device="cuda").manual_seed(11)
    X = torch.randn((16, n), dtype=torch.float64, device="cuda", generator=gen)
    Y, Y64 = torch.empty_like(X), torch.empty_like(X)
    hm.hm_matvec_block(A, X, Y, prec=hm.HM_F64)
    hm.hm_matvec(A, X, Y64, prec=hm.HM_F64)
    torch.cuda.synchronize()
    out = {"workload": "%s (%d panels), leaf %d, 16 right-hand sides on the FP64 master" % (case, n, leaf), "n": n}
    for name, fn in (("df16", lambda: hm.hm_matvec_block(A, X, Y, prec=hm.HM_F64)),
                     ("fp64_x16", lambda: hm.hm_matvec(A, X, Y64, prec=hm.HM_F64))):
        hm.hm_trace_enable(True)
        a, b = _ev(torch), _ev(torch)
        a.record()
        for _ in range(3):
            fn()
        b.record()
        torch.cuda.synchronize()
        hm.hm_trace_enable(False)
        tr = hm.hm_trace_read()
        out[name] = {"ms": a.elapsed_time(b) / 3,
                     "kernels_ms": {k: v[1] / 3 for k, v in sorted(tr.items(), key=lambda kv: -kv[1][1])[:6]}}
    d = torch.linalg.norm(Y - Y64, dim=1) / torch.linalg.norm(Y64, dim=1)
    out["rel_diff_max"] = float(d.max())
    hm.hm_free(A)
    hm.hm_free(tree)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the precision workload's secondary object")
    ap.add_argument("--case", default="large",
                    help="workload: large (default, the headline), precision (the level-7 one-source workload); "
                         "other meshgen recipes run with the one-source step for profiling and parity runs")
    ap.add_argument("--factor-tail-bits", type=int, default=None,
                    help="large workload: keep each block's ACA terms below 2^-bits of its largest in BF16 for the "
                         "16-RHS product (hm_assemble_params.factor_tail_bits; default: the workload's setting)")
    ap.add_argument("--profile-step", action="store_true",
                    help="run exactly one step (no warm-up, no extras) and print its phase times")
    ap.add_argument("--workload", default=None,
                    choices=["batching", "differentiation", "blockmv", "blockmv7", "blockmv_tc", "blockmv8", "blockmv8_tc",
                             "blockmv8_tail", "blockmv_tail", "solve6",
                             "dfmv6", "dfmv8"],
                    help="measure one of the other workloads once and print its numbers (not a bench line)")
    args = ap.parse_args()
    if args.workload:
        print(json.dumps(run_workload(args.workload)))
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count()))
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args, rank, world)))
        return
    import torch
    import paper_1806_11558_gb300 as hm
    from paper_1806_11558_gb300 import build as hb
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    hb.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    if args.case == "large":
        W = dict(LARGE)
        if args.factor_tail_bits is not None:
            W["factor_tail_bits"] = args.factor_tail_bits
        out, extra = run_large(args, world, hm, torch, W=W)
    else:
        W = dict(PRECISION)
        if args.case != "precision":
            import meshgen
            cfg = meshgen.config(args.case)
            W.update(workload="%s (profiling / parity case)" % args.case, case=args.case,
                     panels=int(cfg["T"].shape[0]), leaf_size=cfg["leaf_size"], eta=cfg["eta"],
                     aca_eps=cfg["aca_eps"])
        out, extra = run_single(args, world, hm, torch, W=W, case=args.case)
    if args.profile_step:
        if rank == 0:
            print(json.dumps(out))
        return
    V, T, solve_info = extra
    if args.case == "large" and not args.no_secondary:
        hm.hm_trim()
        mp = {k: solve_info["fma_peaks"][k] for k in ("fp64_tflops", "fp32_tflops", "sm_mhz", "how")}
        out["secondary"] = run_single(args, world, hm, torch, extras=False, fma_peaks=mp)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            v, wall, sample, parts = cpu_oracle_step(solve_info["case"], V, T, solve_info["W"],
                                                     solve_info["n_systems"], solve_info["iters_fp64"])
            out["cpu_baseline"] = {"value": v, "unit": "s", "cores": int(os.environ["OMP_NUM_THREADS"]),
                                   "kind": "oracle", "value_is_estimate": True, "sample": sample, "parts": parts}
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
