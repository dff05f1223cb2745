#!/usr/bin/env python
"""Benchmark: solves/s and factor time at relative residual 1e-8, mixed
(complex64 fronts; the large fronts' block exchanges on the TF32 tensor cores
with two parts per operand, FP32-accurate; the rest FP32) vs FP64
(complex128 fronts) GPU path.

Workload: 2D Helmholtz -lap u - k^2 u = f on [0,1]^2, P2 continuous Galerkin
on a 256 x 256 cell grid (n = 263169, nnz = 3018753), k = 40, first-order
impedance condition (complex symmetric A), Gaussian point source of width
0.02 at a seeded position; box nested dissection with leaf size 64.

One step = one factorization P = L D R (all fronts, Sec. 3.1 / Alg. 3.4) plus
one GMRES solve of A x = b to a float64 true relative residual of 1e-8 with
P^{-1} applied by Algorithm 3.1.  ``value`` is solves per second of the solve
phase (the factorization is reused across solves in practice and is reported
separately as ``factor_ms``, as the metric defines); ``ms_per_step`` includes
both.  Inputs stay resident in HBM; the factor (>= 0.7 GB) exceeds the 129 MB
L2, so every apply streams it from HBM.

Side lines of the same JSON line: ``fp64`` (the comparator), ``ulv``,
``tf32`` (one TF32 part per operand) and ``bf16`` (three BF16 parts per
operand) (other factor variants of the same workload),
``batched`` (64 independent Helmholtz problems x 32 right-hand sides solved
in lockstep; ``--batch-count 0`` skips it) and ``elastic`` (P1 SIPG elastic
waves on 512 x 512 cells, dense, compressed and split-BF16 fronts; ``--elastic-N 0``
skips it).

``--impl reference`` times the FP64 CPU oracle (the only other place this
script runs ``oracle/``) on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "solves/s and factor time at rel. residual 1e-8: mixed vs FP64 GPU path"
WORKLOAD = dict(N=256, p=2, k=40.0, seed=0, leaf=64, tol=1e-8, hss_levels=4, eps_hss=1e-6, beta=64)

# batched side line: independent Helmholtz problems on uneven grids
# (N_x, N_y ~ U{64..256}, wave speed on 8 x 8 macro blocks ~ U[1, 3], 10 points
# per wavelength, impedance), 32 Gaussian sources each, complex64 dense fronts
BATCH = dict(count=64, seed=0, nmin=64, nmax=256, nrhs=32, leaf=64, tol=1e-8)

# elastic side line: P1 SIPG time-harmonic elastic waves (2 displacement
# components, 6 unknowns per triangle), Lame parameters from 16 seeded
# Fourier modes in [1, 4], rho = 1, 8 points per shear wavelength, absorbing
# boundary; tolerance 1e-6; leaf 60, beta 60
ELASTIC = dict(N=512, seed=0, leaf=60, beta=60, tol=1e-6, hss_levels=4)

# C1 side line: 2D Poisson, P1 CG on 64 x 64 cells, homogeneous Dirichlet,
# f ~ U[-1, 1] per node (seed 0), FP64 fronts, leaf 64, HSS eps 1e-6 on the
# levels <= depth - 4, GMRES(30) to 1e-8; also the oracle's compressed factor
# of the same configuration (the like-for-like CPU baseline)
C1 = dict(N=64, seed=0, leaf=64, tol=1e-8, hss_levels=4, eps_hss=1e-6, beta=64, solves=50)

# ncu DRAM traffic of the dominant kernel class, per launch, keyed by the
# sha256 of the source file it was measured on (null once the source changes)
NCU_TRAFFIC = {
    # dram read 585.7 MB + write 11.4 MB per launch
    ("apply", "de495d39c204c920"): 597.1e6,
}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ndhss", choices=["ndhss", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only", choices=["mixed", "fp64", "tf32", "bf16"], help="time one precision only (profiling runs)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer measurement (profiling runs)")
    ap.add_argument("--N", type=int, default=WORKLOAD["N"], help="cells per side (default: the benchmark workload)")
    ap.add_argument("--no-c1", action="store_true", help="skip the C1 Poisson side line")
    ap.add_argument("--batch-count", type=int, default=BATCH["count"],
                    help="problems of the batched side line (0 = skip it)")
    ap.add_argument("--elastic-N", type=int, default=ELASTIC["N"],
                    help="cells per side of the elastic side line (0 = skip it)")
    ap.add_argument("--hss-levels", type=int, default=WORKLOAD["hss_levels"],
                    help="compress fronts on levels <= depth - this (Alg. 3.4); -1 = exact dense fronts")
    return ap.parse_args()


def _workload(N, seed):
    from ndhss_inputs import helmholtz_impedance
    k = WORKLOAD["k"] * N / 256.0
    return helmholtz_impedance(N, WORKLOAD["p"], k, seed=seed)


def _workload_name(P):
    return (f"helmholtz_p2_cg_{P.meta['N']}x{P.meta['N']}_k{P.meta['k']:g}_impedance "
            f"(n={P.n}, nnz={P.A.nnz}, leaf {WORKLOAD['leaf']})")


class Clocks:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.lines = []
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.idx)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.p = None
        return self

    def _read(self):
        for line in self.p.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return pk, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


def _dense_alg_flops(tree):
    """Algorithmic real flops of the dense elimination of every front (the
    LU-based count of the hot-path table: LU of A_ii, the two triangular
    solves for R and L, the Schur product; x4 for complex arithmetic)."""
    import numpy as np
    from paper_2105_07791_gb300 import ndhss
    ni = ndhss.ndhss_tree_export(tree)["node_info"]
    mi, mb = ni[:, 5].astype(float), ni[:, 7].astype(float)
    return float(4.0 * np.sum(2.0 / 3.0 * mi ** 3 + 2.0 * mi ** 2 * mb + 2.0 * mi * mb ** 2))


def _src_sha(name):
    with open(os.path.join(ROOT, "paper_2105_07791_gb300", "csrc", name), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _ulv_summary(r, steps):
    """A side variant of the mixed path measured like the main line: A_ii in
    HSS form with its ULV solve above the switching level, or the front
    updates on the TF32 tensor cores."""
    if not r:
        return None
    ap_ms = sum(v[0] for v in r["applies"]) / steps
    ap_n = sum(v[1] for v in r["applies"]) / steps
    per = r["fstats"]["apply_bytes"]
    dur = ap_ms / max(ap_n, 1)
    return {"solves_per_s": r["solves_per_s"], "factor_ms": r["factor_ms"], "solve_ms": r["solve_ms"],
            "iters": r["iters"], "true_relres": r["true_relres"], "apply_ms": dur, "apply_bytes": per,
            "apply_gbs": per / (dur / 1e3) / 1e9 if dur > 0 else None}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------- replicas (N > 1)
# The path does not shard across GPUs here: every rank factors and solves an
# independent instance (seed + rank); no collective touches the data path.
# Ranks meet only to time: max over ranks of each timed total, and the
# whole-job rate counts every rank's solves.

def replica_seed(rank: int) -> int:
    return WORKLOAD["seed"] + rank


def max_over_ranks(values, device):
    """Element-wise max of a list of floats over the initialised process group
    (identity on one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def whole_job_rate(world: int, steps: int, max_seconds: float) -> float:
    """Solves per second of the whole job: all ranks' solves over the slowest rank's time."""
    return world * steps / max_seconds


# ------------------------------------------------------------------ GPU arm
def run_gpu(a):
    import numpy as np
    import torch

    from paper_2105_07791_gb300 import build, ndhss

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    ndhss.load()
    P = _workload(a.N, replica_seed(rank))              # replicas: an independent instance per rank
    tree = ndhss.ndhss_build_tree(P.coords, P.A.indptr, P.A.indices, WORKLOAD["leaf"])
    M = ndhss.DeviceCSR(P.A)
    b = torch.from_numpy(np.ascontiguousarray(P.b)).cuda()
    x = torch.zeros_like(b)
    stream = torch.cuda.current_stream()
    # FMA rates of this GPU's CUDA cores (the ALU rooflines), before anything is timed
    alu_peaks = {"fp64": ndhss.ndhss_measure_fma_peak(0, stream), "fp32": ndhss.ndhss_measure_fma_peak(1, stream)}

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def fopts(prec, timing=False, ulv=False):
        return ndhss.make_factor_opts(prec=prec, timing=timing, hss_levels=a.hss_levels, eps_hss=WORKLOAD["eps_hss"],
                                      beta=WORKLOAD["beta"], seed=WORKLOAD["seed"], ulv=ulv)

    def one_step(prec, timing, ulv=False):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        f = ndhss.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals, fopts(prec, timing, ulv), stream=stream)
        e1.record(stream)
        st = ndhss.ndhss_gmres(f, M.rowptr, M.col, M.vals, b, x, tol=WORKLOAD["tol"], stream=stream, timing=timing)
        e2.record(stream)
        torch.cuda.synchronize()
        return f, st, e0.elapsed_time(e1), e1.elapsed_time(e2)

    results = {}
    modes = [("mixed", ndhss.NDHSS_FP32, False), ("fp64", ndhss.NDHSS_FP64, False)]
    if not a.only or a.only in ("tf32", "bf16"):
        modes.append(("tf32", ndhss.NDHSS_FP32_TF32, False))
        modes.append(("bf16", ndhss.NDHSS_FP32_BF16, False))
    if a.hss_levels >= 0 and not a.only:
        modes.append(("mixed_ulv", ndhss.NDHSS_FP32, True))
    if a.only:
        modes = [m for m in modes if m[0] == a.only]
    for name, prec, ulv in modes:
        for _ in range(a.warmup):
            f, st, _, _ = one_step(prec, False, ulv)
            del f
        barrier()
        l0 = ndhss.ndhss_kernel_launches()
        fms, sms, its, res, applies = [], [], [], [], []
        fstats = None
        with Clocks(local) as clk:
            tw = time.time()
            for k in range(a.steps):
                f, st, tf, ts = one_step(prec, True, ulv)
                fms.append(tf)
                sms.append(ts)
                its.append(st["iters"])
                res.append(st["true_relres"])
                applies.append((st["apply_ms"], st["napply"], st["spmv_ms"], st["nspmv"]))
                fstats = ndhss.ndhss_factor_stats_get(f)
                del f
            barrier()
            wall = time.time() - tw
        launches = ndhss.ndhss_kernel_launches() - l0
        tot_f, tot_s = max_over_ranks([sum(fms), sum(sms)], "cuda")
        results[name] = dict(kmax=fstats["kmax"], factor_ms=tot_f / a.steps, solve_ms=tot_s / a.steps,
                             solves_per_s=whole_job_rate(world, a.steps, tot_s / 1e3), iters=int(statistics.median(its)),
                             iters_all=its, true_relres=max(res), launches=launches, clocks=clk.summary(),
                             fstats=fstats, applies=applies, wall_s=wall)

    if a.only or a.no_e2e:
        for name, r in results.items():
            if rank == 0:
                print(json.dumps({"profiling_run": name, "factor_ms": r["factor_ms"], "solve_ms": r["solve_ms"],
                                  "iters": r["iters"], "launches": r["launches"], "fstats": r["fstats"]}), flush=True)
        return
    # end-to-end: the same solve through the C ABI with pinned host buffers
    f = ndhss.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals, fopts(ndhss.NDHSS_FP32), stream=stream)
    bh = torch.from_numpy(np.ascontiguousarray(P.b)).pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    bn, xn = bh.numpy(), xh.numpy()
    for _ in range(a.warmup):
        ndhss.ndhss_gmres(f, M.rowptr, M.col, M.vals, bn, xn, tol=WORKLOAD["tol"], stream=stream)
    barrier()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        ndhss.ndhss_gmres(f, M.rowptr, M.col, M.vals, bn, xn, tol=WORKLOAD["tol"], stream=stream)
    barrier()
    e2e_s = max_over_ranks([time.perf_counter() - t0], "cuda")[0]
    relres_e2e = float(np.linalg.norm(P.b - P.A @ xn) / np.linalg.norm(P.b))
    del f

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    mx, fp = results["mixed"], results["fp64"]
    pk, pk_kind = _peaks()
    # roofline of the kernel behind `value` (solves/s; the metric excludes the
    # factorization): the apply, one persistent launch per application, timed
    # live by CUDA events on the launching stream around every application
    fs = mx["fstats"]
    cls_ms = fs["class_ms"]
    ap_ms = sum(v[0] for v in mx["applies"]) / a.steps
    ap_n = sum(v[1] for v in mx["applies"]) / a.steps
    sp_ms = sum(v[2] for v in mx["applies"]) / a.steps
    per = fs["apply_bytes"]
    dur_ms = ap_ms / max(ap_n, 1)
    ach = per / (dur_ms / 1e3) / 1e9
    roof = {"kernel": "apply_dataflow_kernel (Alg. 3.1: up-sweep, diagonal, down-sweep as one persistent launch)",
            "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": ach / pk["hbm_gbs"],
            "traffic": NCU_TRAFFIC.get(("apply", _src_sha("apply.cu"))), "peak_kind": f"hbm_gbs, {pk_kind}",
            "algorithmic_bytes_per_launch": per, "avg_launch_ms": dur_ms,
            "solve_share": ap_ms / mx["solve_ms"] if mx["solve_ms"] > 0 else None}
    # the factorization's dominant class, for the factor-time half of the metric
    dom = max(cls_ms, key=cls_ms.get)
    froof = {"class": dom, "ms_per_factor": cls_ms[dom], "launches": fs["class_launches"][dom],
             "share_of_factor": cls_ms[dom] / mx["factor_ms"] if mx["factor_ms"] > 0 else None}
    # TF32 dense tensor peak: the measured BF16 burst times the nominal TF32 /
    # BF16 ratio (1.1 / 2.25 PFLOP/s); a product split into two TF32 parts takes
    # three MMAs, so FP32-accurate products run at a third of it
    tf32_peak = pk["bf16_tflops"] * 1.1 / 2.25
    dense_ms = sum(cls_ms.get(k, 0.0) for k in ("panel", "prep", "update", "finalize", "tensor"))
    alg = _dense_alg_flops(tree)
    froof["dense_elimination"] = {
        "bound": "tensor", "unit": "TFLOP/s", "algorithmic_flops": alg, "ms_per_factor": dense_ms,
        "achieved": alg / (dense_ms / 1e3) / 1e12 if dense_ms > 0 else None, "peak": tf32_peak / 3,
        "peak_kind": f"TF32 dense ({pk_kind} bf16 x 1.1/2.25) / 3 (two-part split: three MMAs per product)",
        "algorithmic": "LU-based count per complex front: 8/3 m_i^3 + 8 m_i^2 m_b + 8 m_i m_b^2"}
    if froof["dense_elimination"]["achieved"]:
        froof["dense_elimination"]["frac"] = froof["dense_elimination"]["achieved"] / (tf32_peak / 3)
    if dom == "compress":
        froof.update(bound="latency (per-round row-ID pivot chains of the HSS levels, one dependent launch each)")
    # the other hot kernels against the bound that limits them: the FP64 and
    # FP32 FMA rates measured on this GPU in this run (the library's
    # independent-FMA-chain kernel), HBM from the measured peaks
    fp64_peak, fp32_peak = alu_peaks["fp64"], alu_peaks["fp32"]
    n_sp = sum(v[3] for v in mx["applies"]) / a.steps
    sp_bytes = 20 * P.A.nnz + 36 * P.n
    cplx_entries = int(np.count_nonzero(np.imag(P.A.data))) if np.iscomplexobj(P.A.data) else 0
    sp_flops = 4.0 * (P.A.nnz - cplx_entries) + 8.0 * cplx_entries
    sp_one = sp_ms / max(n_sp, 1)
    krl = [
        dict(roof, kernel="apply_dataflow_kernel"),
        {"kernel": "gm_spmv_kernel (FP64 CSR, complex128; inside the GMRES solves)", "bound": "hbm", "unit": "GB/s",
         "achieved": sp_bytes / (sp_one / 1e3) / 1e9 if sp_one > 0 else None, "peak": pk["hbm_gbs"],
         "peak_kind": f"hbm_gbs, {pk_kind}", "algorithmic": "20 B per entry (value, column) + 36 B per row (row "
         "pointer, x, y), x read once", "algorithmic_bytes_per_launch": sp_bytes, "avg_launch_ms": sp_one,
         "fp64": {"flops": sp_flops, "achieved_tflops": sp_flops / (sp_one / 1e3) / 1e12 if sp_one > 0 else None,
                  "peak_tflops": fp64_peak, "note": "4 flops per real entry, 8 per complex entry; FP64 FMA rate "
                  "measured in this run"}},
        {"kernel": "gemm_update_kernel (FP32 SIMT rank-kb exchange steps: small fronts, slabs of the large ones)",
         "bound": "alu", "unit": "TFLOP/s",
         "achieved": fs["update_flops"] / (cls_ms["update"] / 1e3) / 1e12 if cls_ms.get("update") else None,
         "peak": fp32_peak, "peak_kind": "FP32 FMA rate measured in this run",
         "algorithmic": "8 m x (columns exchanged) x kb flops per front and panel"},
        {"kernel": "tc_gemm_kernel (tcgen05 + TMA rank-128 block exchanges, two TF32 parts per operand; class "
                   "time includes the operand packing)", "bound": "tensor", "unit": "TFLOP/s",
         "achieved": fs["tc_flops"] / (cls_ms["tensor"] / 1e3) / 1e12 if cls_ms.get("tensor") else None,
         "peak": tf32_peak / 3, "peak_kind": f"TF32 dense ({pk_kind} bf16 x 1.1/2.25) / 3 MMAs per product",
         "algorithmic": "8 m (m - w) w flops per front and outer block of w pivots"},
    ]
    for k in krl:
        if k.get("achieved") is not None and k.get("peak"):
            k["frac"] = k["achieved"] / k["peak"]
    line = {
        "metric": METRIC,
        "value": mx["solves_per_s"],
        "unit": "solves/s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": mx["factor_ms"] + mx["solve_ms"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "c64 fronts (fp32) / c128 Krylov (fp64)",
        "data": "synthetic",
        "config": {"workload": _workload_name(P), "rhs_per_step": 1, "tol": WORKLOAD["tol"],
                   "compression": (f"HSS on levels <= depth - {a.hss_levels}, eps {WORKLOAD['eps_hss']:g}, beta "
                                   f"{WORKLOAD['beta']}" if a.hss_levels >= 0 else "off (exact dense fronts)"), "l2": "inputs exceed L2 (factor streamed from HBM)",
                   "parallelism": f"replicas x{world}"},
        "factor_ms": mx["factor_ms"],
        "solve_ms": mx["solve_ms"],
        "iters": mx["iters"],
        "kmax": fs["kmax"],
        "apply_bytes": fs["apply_bytes"],
        "true_relres": mx["true_relres"],
        "fp64": {"solves_per_s": fp["solves_per_s"], "factor_ms": fp["factor_ms"], "solve_ms": fp["solve_ms"],
                 "iters": fp["iters"], "true_relres": fp["true_relres"], "kmax": fp["kmax"],
                 "apply_bytes": fp["fstats"]["apply_bytes"]},
        "mixed_over_fp64": {"solves_per_s": mx["solves_per_s"] / fp["solves_per_s"],
                            "factor_speedup": fp["factor_ms"] / mx["factor_ms"]},
        "ulv": _ulv_summary(results.get("mixed_ulv"), a.steps),
        "tf32": _ulv_summary(results.get("tf32"), a.steps),
        "bf16": _ulv_summary(results.get("bf16"), a.steps),
        "apply_gbs": fs["apply_bytes"] / (ap_ms / max(ap_n, 1) / 1e3) / 1e9,
        "e2e": {"value": whole_job_rate(world, a.steps, e2e_s), "unit": "solves/s", "h2d_bytes_per_step": int(P.b.nbytes),
                "d2h_bytes_per_step": int(xn.nbytes), "true_relres": relres_e2e},
        "gpu_launches": mx["launches"],
        "roofline": roof,
        "factor_roofline": froof,
        "kernel_rooflines": krl,
        "alu_peaks_tflops": alu_peaks,
        "spmv_ms_per_solve": sp_ms,
        "factor_kernel_ms": {k: round(v, 3) for k, v in cls_ms.items()},
        "clocks": mx["clocks"],
    }
    if a.batch_count > 0:
        line["batched"] = batched_line(a, ndhss, torch, stream)
        b = line["batched"]
        krl.append({"kernel": "mapply_kernel (batched 32-column apply)", "bound": "alu", "unit": "TFLOP/s",
                    "achieved": b["apply_multi_tflops"], "peak": fp32_peak,
                    "peak_kind": "FP32 FMA rate measured in this run",
                    "frac": b["apply_multi_tflops"] / fp32_peak, "algorithmic": "8 x 32 flops per stored element"})
    if a.elastic_N > 0:
        line["elastic"] = elastic_line(a, ndhss, torch, stream)
    if not a.no_c1:
        line["c1"] = c1_line(a, ndhss, torch, stream)
    if not a.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(P)
        if "c1" in line:
            line["cpu_baseline"]["like_for_like_c1"] = c1_oracle()
            line["c1"]["gpu_over_oracle"] = line["c1"]["solves_per_s"] / line["cpu_baseline"]["like_for_like_c1"]["solves_per_s"]
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _mapply_tiles():
    """The committed tile-shape table of the 32-column apply (autotune.py)."""
    from paper_2105_07791_gb300 import autotune
    return autotune.current_table()


def batched_line(a, ndhss, torch, stream):
    """The batched workload: every step factors the forest of all problems
    (one call, complex64 dense fronts) and solves problems x 32 right-hand
    sides in lockstep to a true relative residual of 1e-8 each."""
    import numpy as np

    from ndhss_inputs import helmholtz_batch

    t0 = time.time()
    probs = helmholtz_batch(a.batch_count, BATCH["seed"], nmin=BATCH["nmin"], nmax=BATCH["nmax"], nsrc=BATCH["nrhs"])
    tree = ndhss.ndhss_build_tree_batched([(P.coords, P.A.indptr, P.A.indices) for P in probs], BATCH["leaf"])
    A, off = ndhss.batch_csr([P.A for P in probs])
    setup_s = time.time() - t0
    M = ndhss.DeviceCSR(A)
    n = A.shape[0]
    Bh = np.zeros((BATCH["nrhs"], n), dtype=np.complex128)
    for s, P in enumerate(probs):
        Bh[:, off[s]:off[s + 1]] = P.b.T
    B = torch.from_numpy(Bh).cuda()
    X = torch.zeros_like(B)
    opts = ndhss.make_factor_opts(prec=ndhss.NDHSS_FP32, hss_levels=-1)

    def step():
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        f = ndhss.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals, opts, stream=stream)
        e1.record(stream)
        st = ndhss.ndhss_gmres_batched(f, M.rowptr, M.col, M.vals, off, B, X, tol=BATCH["tol"], stream=stream)
        e2.record(stream)
        torch.cuda.synchronize()
        return f, st, e0.elapsed_time(e1), e1.elapsed_time(e2)

    for _ in range(max(1, min(a.warmup, 2))):
        f, st, _, _ = step()
        del f
    steps = max(1, min(a.steps, 5))
    fms, sms = [], []
    l0 = ndhss.ndhss_kernel_launches()
    for _ in range(steps):
        f, st, tf, ts = step()
        fms.append(tf)
        sms.append(ts)
    launches = (ndhss.ndhss_kernel_launches() - l0) // steps
    flat = [d for row in st for d in row]
    # the 32-column apply alone (events around ndhss_apply_multi on interleaved vectors)
    Xi = torch.randn((n, BATCH["nrhs"]), dtype=torch.complex128, device="cuda")
    Yi = torch.empty_like(Xi)
    ndhss.ndhss_apply_multi(f, Xi, Yi, stream=stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(5):
        ndhss.ndhss_apply_multi(f, Xi, Yi, stream=stream)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ap_ms = ev[0].elapsed_time(ev[1]) / 5
    fs = ndhss.ndhss_factor_stats_get(f)
    del f
    # algorithmic work of one 32-column apply: every stored front element of
    # the first m_i columns and of R read once, 32 complex multiply-adds each
    ni = ndhss.ndhss_tree_export(tree)["node_info"]
    mi, mb = ni[:, 5].astype(np.int64), ni[:, 7].astype(np.int64)
    elems = int(np.sum(mi * (mi + mb) + mi * mb))
    flops = 8.0 * BATCH["nrhs"] * elems
    nsolve = len(probs) * BATCH["nrhs"]
    solve_ms = sum(sms) / steps
    # the same batch on a compressed forest factor (HSS on the levels <= depth - 4
    # of every problem's tree, eps 1e-6, beta 64): one warm-up, one timed step
    copts = ndhss.make_factor_opts(prec=ndhss.NDHSS_FP32, hss_levels=4, eps_hss=1e-6, beta=64)
    fc = ndhss.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals, copts, stream=stream)
    del fc
    X.zero_()
    c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    c0.record(stream)
    fc = ndhss.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals, copts, stream=stream)
    c1.record(stream)
    stc = ndhss.ndhss_gmres_batched(fc, M.rowptr, M.col, M.vals, off, B, X, tol=BATCH["tol"], stream=stream)
    c2.record(stream)
    torch.cuda.synchronize()
    fsc = ndhss.ndhss_factor_stats_get(fc)
    del fc
    flc = [d for row in stc for d in row]
    compressed = {"factor_ms": c0.elapsed_time(c1), "solve_ms": c1.elapsed_time(c2),
                  "solves_per_s": nsolve / (c1.elapsed_time(c2) / 1e3), "kmax": fsc["kmax"],
                  "factor_bytes": fsc["factor_bytes"], "iters_median": int(statistics.median(d["iters"] for d in flc)),
                  "iters_max": max(d["iters"] for d in flc), "true_relres_max": max(d["true_relres"] for d in flc),
                  "converged": all(d["converged"] for d in flc)}
    return {"workload": f"helmholtz_macro_p1 x{len(probs)} (grids {BATCH['nmin']}..{BATCH['nmax']}, "
                        f"c on 8x8 macro blocks U[1,3], 10 ppw, impedance)",
            "problems": len(probs), "rhs_per_problem": BATCH["nrhs"], "n_total": int(n), "nnz_total": int(A.nnz),
            "solves_per_step": nsolve, "steps": steps, "factor_ms": sum(fms) / steps, "solve_ms": solve_ms,
            "solves_per_s": nsolve / (solve_ms / 1e3), "iters_median": int(statistics.median(d["iters"] for d in flat)),
            "iters_max": max(d["iters"] for d in flat), "true_relres_max": max(d["true_relres"] for d in flat),
            "converged": all(d["converged"] for d in flat), "gpu_launches_per_step": int(launches),
            "factor_bytes": fs["factor_bytes"], "apply_multi_ms": ap_ms,
            "apply_multi_tflops": flops / (ap_ms / 1e3) / 1e12, "apply_multi_flops": flops,
            "host_setup_s": setup_s, "compressed": compressed, "mapply_tiles": _mapply_tiles()}


def elastic_line(a, ndhss, torch, stream):
    """The elastic workload: per variant (complex64 fronts: FP32 arithmetic
    dense and compressed, and the front update with BF16 tensor-core operands)
    one warm-up factorization, then one timed factorization and one GMRES
    solve to a true relative residual of 1e-6."""
    import numpy as np

    from ndhss_inputs.elastic import elastic_sipg

    t0 = time.time()
    P = elastic_sipg(a.elastic_N, seed=ELASTIC["seed"])
    tree = ndhss.ndhss_build_tree(P.coords, P.A.indptr, P.A.indices, ELASTIC["leaf"])
    setup_s = time.time() - t0
    M = ndhss.DeviceCSR(P.A)
    b = torch.from_numpy(np.ascontiguousarray(P.b)).cuda()
    out = {"workload": f"elastic_sipg_p1_{a.elastic_N}x{a.elastic_N} (n={P.n}, nnz={P.A.nnz}, "
                       f"omega={P.meta['omega']:.1f}, leaf {ELASTIC['leaf']}, beta {ELASTIC['beta']})",
           "tol": ELASTIC["tol"], "host_setup_s": setup_s}
    for name, hl, prec in (("dense", -1, ndhss.NDHSS_FP32), ("compressed", ELASTIC["hss_levels"], ndhss.NDHSS_FP32),
                           ("dense_bf16", -1, ndhss.NDHSS_FP32_BF16)):
        opts = ndhss.make_factor_opts(prec=prec, hss_levels=hl, eps_hss=1e-6, beta=ELASTIC["beta"])
        f = ndhss.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals, opts, stream=stream)
        del f
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        x = torch.zeros_like(b)
        e0.record(stream)
        f = ndhss.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals, opts, stream=stream)
        e1.record(stream)
        st = ndhss.ndhss_gmres(f, M.rowptr, M.col, M.vals, b, x, tol=ELASTIC["tol"], timing=True, stream=stream)
        e2.record(stream)
        torch.cuda.synchronize()
        fs = ndhss.ndhss_factor_stats_get(f)
        del f
        out[name] = {"factor_ms": e0.elapsed_time(e1), "solve_ms": e1.elapsed_time(e2),
                     "solves_per_s": 1e3 / e1.elapsed_time(e2), "iters": st["iters"], "converged": st["converged"],
                     "true_relres": st["true_relres"], "apply_ms": st["apply_ms"] / max(st["napply"], 1),
                     "apply_bytes": fs["apply_bytes"], "factor_bytes": fs["factor_bytes"], "kmax": fs["kmax"],
                     "apply_gbs": fs["apply_bytes"] / (st["apply_ms"] / max(st["napply"], 1) / 1e3) / 1e9
                     if st["apply_ms"] > 0 else None}
    return out


def _c1_problem():
    from ndhss_inputs import poisson_dirichlet
    return poisson_dirichlet(C1["N"], seed=C1["seed"])


def c1_line(a, ndhss, torch, stream):
    """C1: the Poisson configuration, FP64 fronts with HSS compression;
    factor time (three factorizations after a warm-up, mean), then C1["solves"]
    GMRES solves to 1e-8 timed together (solves/s), and one solve with the
    apply timed for its GB/s."""
    import numpy as np

    P = _c1_problem()
    tree = ndhss.ndhss_build_tree(P.coords, P.A.indptr, P.A.indices, C1["leaf"])
    M = ndhss.DeviceCSR(P.A)
    b = torch.from_numpy(np.ascontiguousarray(P.b)).cuda()
    opts = ndhss.make_factor_opts(prec=ndhss.NDHSS_FP64, hss_levels=C1["hss_levels"], eps_hss=C1["eps_hss"],
                                  beta=C1["beta"], seed=0)
    f = ndhss.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals, opts, stream=stream)
    del f
    torch.cuda.synchronize()
    fms = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f = ndhss.ndhss_factor(tree, M.vtype, M.rowptr, M.col, M.vals, opts, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        fms.append(e0.elapsed_time(e1))
        if len(fms) < 3:
            del f
    x = torch.zeros_like(b)
    for _ in range(3):
        x.zero_()
        ndhss.ndhss_gmres(f, M.rowptr, M.col, M.vals, b, x, tol=C1["tol"], stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(C1["solves"]):
        x.zero_()
        st = ndhss.ndhss_gmres(f, M.rowptr, M.col, M.vals, b, x, tol=C1["tol"], stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    solve_ms = e0.elapsed_time(e1) / C1["solves"]
    x.zero_()
    stt = ndhss.ndhss_gmres(f, M.rowptr, M.col, M.vals, b, x, tol=C1["tol"], timing=True, stream=stream)
    fs = ndhss.ndhss_factor_stats_get(f)
    xs = x.cpu().numpy()
    relres = float(np.linalg.norm(P.b - P.A @ xs) / np.linalg.norm(P.b))
    ap_ms = stt["apply_ms"] / max(stt["napply"], 1)
    return {"workload": f"poisson_p1_cg_{C1['N']}x{C1['N']}_dirichlet (n={P.n}, nnz={P.A.nnz}, leaf {C1['leaf']})",
            "dtype": "f64 fronts, f64 Krylov",
            "compression": f"HSS on levels <= depth - {C1['hss_levels']}, eps {C1['eps_hss']:g}, beta {C1['beta']}",
            "factor_ms": statistics.mean(fms), "solve_ms": solve_ms, "solves_per_s": 1e3 / solve_ms,
            "iters": st["iters"], "true_relres": relres, "kmax": fs["kmax"], "apply_ms": ap_ms,
            "apply_bytes": fs["apply_bytes"],
            "apply_gbs": fs["apply_bytes"] / (ap_ms / 1e3) / 1e9 if ap_ms > 0 else None,
            "note": "a 4k-unknown problem: every kernel is launch- and latency-bound, not bandwidth-bound"}


def c1_oracle():
    """The oracle's compressed factor of C1 (the same preconditioner as the
    GPU's C1 line: FP64, same tree, eps, beta, Philox streams), timed on the
    host cores: tree + factor once, then GMRES solves for about 2 s."""
    from oracle.gmres import gmres
    from oracle.hss import apply_compressed, factor_compressed
    from oracle.tree import build_tree
    P = _c1_problem()
    t0 = time.perf_counter()
    T = build_tree(P.coords, P.A.indptr, P.A.indices, C1["leaf"])
    t1 = time.perf_counter()
    fac = factor_compressed(T, P.A, hss_levels=C1["hss_levels"], eps=C1["eps_hss"], beta=C1["beta"], k0=32, r=16,
                            seed=0)
    t2 = time.perf_counter()
    n = 0
    t3 = time.perf_counter()
    while True:
        r = gmres(P.A, P.b, lambda v: apply_compressed(fac, v), tol=C1["tol"])
        n += 1
        if time.perf_counter() - t3 > 2.0:
            break
    ts = (time.perf_counter() - t3) / n
    return {"value": 1.0 / ts, "solves_per_s": 1.0 / ts, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"C1 with the oracle's compressed FP64 factor (the GPU C1 line's preconditioner): {n} GMRES solves "
                      f"(tol 1e-8, {r.iters} it) after one factorization",
            "factor_s": t2 - t1, "tree_s": t1 - t0, "iters": r.iters, "kmax": fac.kmax}


# ------------------------------------------------------------- CPU oracle
def _oracle_setup(P):
    from oracle.frontal import apply_inverse, factor_dense
    from oracle.tree import build_tree
    t0 = time.perf_counter()
    T = build_tree(P.coords, P.A.indptr, P.A.indices, WORKLOAD["leaf"])
    t1 = time.perf_counter()
    fac = factor_dense(T, P.A)
    t2 = time.perf_counter()
    return fac, apply_inverse, t1 - t0, t2 - t1


def cpu_baseline(P):
    """The FP64 oracle as it stands, on the host cores: factor once, then one solve."""
    from oracle.gmres import gmres
    fac, apply_inverse, t_tree, t_fac = _oracle_setup(P)
    t0 = time.perf_counter()
    r = gmres(P.A, P.b, lambda v: apply_inverse(fac, v), tol=WORKLOAD["tol"])
    ts = time.perf_counter() - t0
    t0 = time.perf_counter()
    apply_inverse(fac, P.b)
    t_apply = time.perf_counter() - t0
    return {"value": 1.0 / ts, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"one GMRES solve (tol 1e-8, {r.iters} it) on the full workload with the oracle's "
                       f"dense FP64 factor; factor built once beforehand in {t_fac:.1f} s (tree {t_tree:.1f} s), "
                       "not counted, like the GPU value"),
            "factor_s": t_fac, "tree_s": t_tree, "apply_ms": 1e3 * t_apply, "iters": r.iters}


def run_reference(a):
    world, rank, _ = _dist()
    if rank != 0:
        return
    P = _workload(a.N, WORKLOAD["seed"])
    from oracle.gmres import gmres
    fac, apply_inverse, t_tree, t_fac = _oracle_setup(P)
    for _ in range(a.warmup):
        gmres(P.A, P.b, lambda v: apply_inverse(fac, v), tol=WORKLOAD["tol"])
    t0 = time.perf_counter()
    its = []
    for _ in range(a.steps):
        r = gmres(P.A, P.b, lambda v: apply_inverse(fac, v), tol=WORKLOAD["tol"])
        its.append(r.iters)
    ts = time.perf_counter() - t0
    val = a.steps / ts
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "solves/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * ts / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64/c128", "data": "synthetic",
            "config": {"workload": _workload_name(P), "rhs_per_step": 1, "tol": WORKLOAD["tol"]},
            "factor_ms": 1e3 * t_fac, "iters": int(statistics.median(its)),
            "cpu_baseline": {"value": val, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": ("each step one GMRES solve on the full workload with the oracle's dense "
                                        f"FP64 factor, built once beforehand in {t_fac:.1f} s")},
            "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_gpu(a)


if __name__ == "__main__":
    main()
