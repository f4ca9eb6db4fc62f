"""Benchmark: seconds for one PCG solve to relative residual 1e-8 of the 350^3
diffusion problem with the nested twisted filtering preconditioner
(arXiv 1909.09771) on one GB300, setup included.

A step = one full pass of the hot path over one input: the learned filter's
inference on kappa, operator assembly, preconditioner setup (FP32 factors),
and the flexible-CG solve to rtol, inputs resident in HBM.  The metric
compares that form with the plain FP64 one (FP64 factors, rowsum filter, same
preconditioner and tolerance), which the same run times once on the same GPU
and reports as config.fp64_rowsum.  `e2e` repeats the step through the public
API from pinned host buffers (kappa and b copied in, x copied out inside the
timed region).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload grf350|layered128|blocks32|batched|paper<T>_<n>]
                  [--precision fp32|fp64|bf16] [--precond combo|ntd] [--rtol R]
                  [--filter learned|rowsum] [--fp64-steps F]

paper<T>_<n> (T = 1, 2, 3; e.g. paper1_350) is the paper's own test matrix of
type T on n^3 (Sec. IV, Table I); compare with --rtol 1e-7 or 1e-10.

--impl reference times the CPU oracle (plain C, FP64, one core) on a bounded
sample of the same workload.  Under torchrun (N > 1) the ranks solve
independent replicas (the single-instance solve does not shard) and rank 0
prints the aggregate; the batched workload shards its instance list.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PCG s to rel-res 1e-8 at 350^3 (learned+FP32 vs plain FP64); apply GB/s vs HBM"
RTOL = 1e-8
L2_BYTES = 129e6
MAXIT = 1000

# Algorithmic bytes per unknown of one B_NTD apply: 2 sweeps x 4 factor arrays
# (l1, 1/M, l2, l3) in the storage precision + 4 FP64 vector passes (read r,
# write y, read y, write z): 96 / 64 / 48 bytes for FP64 / FP32 / BF16 factors.
NTD_BYTES = {"fp64": 2 * 4 * 8 + 4 * 8, "fp32": 2 * 4 * 4 + 4 * 8, "bf16": 2 * 4 * 2 + 4 * 8}
# SpMV fused with (p, q): p 8 + q 8 + 4 FP64 bands 32 bytes per unknown, and 8 FP64
# operations on the FMA pipe per unknown (d x, six couplings, the (p, q) term).
SPMV_BYTES = 48
SPMV_FP64_OPS = 8
# FP64 FMA-pipe operations per second of the part: 152 SMs x 2 FP64 FMA per clock x 2070 MHz
# (the nominal 1.25 TFLOP/s FP64 at the maximum SM clock).
FP64_OPS_PEAK = 152 * 2 * 2.07e9


def make_workload(name, seed=0):
    from paper_1909_09771_gb300 import inputs as I
    if name == "grf350":
        return I.workload_grf(seed=seed, n=350)
    if name == "layered128":
        return I.workload_layered128(seed=seed)
    if name == "blocks32":
        return I.workload_blocks32(seed=seed)
    if name.startswith("grf"):
        return I.workload_grf(seed=seed, n=int(name[3:]))
    if name.startswith("paper"):  # paper<type>_<n>: the paper's test problems
        kind, n = name[5:].split("_")
        return I.workload_paper(int(kind), int(n))
    raise ValueError(name)


def describe(name):
    return {
        "grf350": "350^3 cells (42.875M unknowns), unit cube, Dirichlet z-faces, Neumann x/y; "
                  "kappa = 10^(3 g), g seeded Gaussian random field (corr. length 0.1) clipped to "
                  "[-1,1] (contrast 10^6); b ~ N(0,1)",
        "layered128": "128^3, 16 z-layers kappa 1/1e6 with eight 16^3 inclusions 1e-3; b = h^3",
        "blocks32": "32^3, kappa 10^e on 4x4x4 blocks, e in [-3,3]; b ~ N(0,1)",
        "batched": "64 instances, nx,ny,nz ~ U[48,160] each (uneven), kappa 10^e on 8x8x8 blocks, "
                   "e in [-3,3], Dirichlet z-faces, Neumann x/y; 4 right-hand sides N(0,1) each "
                   "(256 solves per step)",
    }.get(name, paper_describe(name))


def paper_describe(name):
    if not name.startswith("paper"):
        return name
    kind, n = name[5:].split("_")
    what = {"1": "skyscrapers with checkerboard jumps, kappa 10^3 ([10 y] + 1) on even blocks, else 1",
            "2": "kappa 10^3 on the shell 1/(2 sqrt 2) <= |x - c| <= 1/2, else 1",
            "3": "Poisson, kappa = 1"}[kind]
    return (f"the paper's test matrix type {kind} (Sec. IV): {n}^3 unit cube, Dirichlet on all faces, "
            f"{what}; b = h^3")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self):
        rows = [r for r in csv.reader(io.StringIO(getattr(self, "out", ""))) if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i]
                          and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_seed(workload, seed, rank):
    """Seed of rank `rank`'s replica of a single-instance workload: every rank
    solves its own independent problem (the solve does not shard), so the
    ranks' inputs must differ.  (The batched workload is not replicated: its
    one instance list is partitioned, see lpt_partition.)"""
    return seed + rank


def lpt_partition(sizes, nranks):
    """Partition instances over ranks by longest-processing-time-first on
    their size (n = nx ny nz, which sets an instance's setup work and its
    per-iteration sweep and vector work): instances in decreasing size, each
    to the rank with the smallest load so far (the lowest rank on ties).
    Deterministic; returns every rank's instance indices in increasing order.
    Its load is within one instance of the best balance (Graham's bound:
    max load <= mean load + largest instance)."""
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    load = [0] * nranks
    parts = [[] for _ in range(nranks)]
    for i in order:
        r = min(range(nranks), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += sizes[i]
    return [sorted(p) for p in parts]


def merge_pair_stats(local_stats, local_instances, nrhs, count, world_size):
    """Every rank's per-pair statistics in global pair order (instance i,
    right-hand side j -> i * nrhs + j), gathered to all ranks.  Only these
    small host records are exchanged; no solver data crosses ranks."""
    if world_size <= 1:
        return list(local_stats)
    import torch.distributed as dist
    objs = [None] * world_size
    dist.all_gather_object(objs, (list(local_instances), list(local_stats)))
    out = [None] * (count * nrhs)
    for insts, stats in objs:
        for j, i in enumerate(insts):
            for r in range(nrhs):
                out[i * nrhs + r] = stats[j * nrhs + r]
    assert all(v is not None for v in out)
    return out


def max_over_ranks(values, device, world_size):
    """Element-wise maximum over ranks of a list of floats (the job's time is
    its slowest rank's)."""
    if world_size <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def solve_step(ffp, grid, bc, precision, precond, work, net, t_buf, rtol, stream, schur="newton"):
    """One pass of the hot path on resident inputs: the learned filter's
    inference (if any), assembly + setup, and the flexible-CG solve to rtol.
    Returns a function step(kappa, b, x, marks) -> stats."""
    import torch

    def step(kap, rhs, xout, marks=None):
        if marks is not None:
            marks.append([torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)])
            marks[-1][0].record(stream)
        t = net.forward(grid, kap, batch=1, t=t_buf) if net is not None else None
        P = ffp.Preconditioner(grid, kap, bc, precision, precond=precond, workspace=work, t=t,
                               schur=schur)
        if marks is not None:
            marks[-1][1].record(stream)
        xout.zero_()
        _, st = P.solve(rhs, x=xout, rtol=rtol, maxit=MAXIT, check=False)
        P.close()
        return st
    return step


def timed_steps(step, kappa, b, x, steps, local):
    """`steps` device-timed steps (CUDA events on the launching stream, a
    synchronise on both sides); returns (ms per step, setup ms per step, stats,
    clock summary)."""
    import torch
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats, marks = [], []
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(steps):
            stats.append(step(kappa, b, x, marks))
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    setup_ms = sum(m0.elapsed_time(m1) for m0, m1 in marks) / len(marks)
    return ms, setup_ms, stats, clk.summary()


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1909_09771_gb300 import ffp

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = make_workload(args.workload, seed=replica_seed(args.workload, args.seed, rank))
    grid, bc = w["grid"], w["bc"]
    n = int(w["kappa"].size)
    kappa_h = torch.from_numpy(w["kappa"]).pin_memory()
    b_h = torch.from_numpy(w["b"]).pin_memory()
    x_h = torch.empty(n, dtype=torch.float64).pin_memory()
    kappa = kappa_h.to(dev)
    b = b_h.to(dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    # workspace allocated once and reused by every step (the library never allocates)
    wsb = ffp.workspace_bytes(grid, args.precision)
    work = torch.empty(wsb, dtype=torch.uint8, device=dev)

    net, t_buf = None, None
    if args.filter == "learned":
        from paper_1909_09771_gb300 import learned as LF
        net = LF.load_weights(args.weights, device=dev)
        t_buf = torch.empty(n, dtype=torch.float64, device=dev)
    step = solve_step(ffp, grid, bc, args.precision, args.precond, work, net, t_buf, args.rtol, stream,
                      args.schur)

    def barrier():
        if ws > 1:
            dist.barrier()

    for _ in range(args.warmup):
        step(kappa, b, x)
    torch.cuda.synchronize()
    # ---- device-resident timed region
    barrier()
    ms, setup_ms, stats, clocks = timed_steps(step, kappa, b, x, args.steps, local)
    barrier()
    # ---- end to end through the public API with host buffers
    e2e_steps = max(1, min(args.steps, args.e2e_steps))  # the line always carries an end-to-end number
    e2 = []
    barrier()
    torch.cuda.synchronize()
    for _ in range(e2e_steps):
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        kd = kappa_h.to(dev, non_blocking=True)
        bd = b_h.to(dev, non_blocking=True)
        step(kd, bd, x)
        x_h.copy_(x, non_blocking=True)
        t1.record(stream)
        torch.cuda.synchronize()
        e2.append(t0.elapsed_time(t1))
    barrier()
    e2e_ms = sum(e2) / len(e2)
    ms, e2e_ms = max_over_ranks([ms, e2e_ms], dev, ws)
    st = stats[-1]
    ok = all(s["status"] == 0 and s["rel_res_true"] < args.rtol for s in stats)

    # ---- the plain FP64 form on the same GPU: FP64 factors, rowsum filter, same
    # preconditioner and tolerance (one GPU only: the comparison the metric names)
    fp64 = None
    if args.fp64_steps > 0 and ws == 1 and not (args.precision == "fp64" and net is None):
        del work
        torch.cuda.empty_cache()
        work64 = torch.empty(ffp.workspace_bytes(grid, "fp64"), dtype=torch.uint8, device=dev)
        step64 = solve_step(ffp, grid, bc, "fp64", args.precond, work64, None, None, args.rtol, stream,
                            args.schur)
        # warm-up: one setup and one preconditioner application load the FP64 kernels
        P = ffp.Preconditioner(grid, kappa, bc, "fp64", precond=args.precond, workspace=work64,
                               schur=args.schur)
        P.apply(b)
        P.close()
        ms64, setup64, stats64, clocks64 = timed_steps(step64, kappa, b, x, args.fp64_steps, local)
        s64 = stats64[-1]
        fp64 = {"s": ms64 / 1e3, "setup_s": setup64 / 1e3, "iters": s64["iters"],
                "rel_res_true": s64["rel_res_true"], "cond_est": s64["cond_est"],
                "converged": all(s["status"] == 0 and s["rel_res_true"] < args.rtol for s in stats64),
                "steps": args.fp64_steps, "warmup": "one setup + one apply (loads the FP64 kernels)",
                "ms_per_apply_ntd": s64["ntd_ms"] / max(s64["napply"], 1),
                "clocks": clocks64}
        del work64

    peak, peak_kind = load_peaks()
    ntd_per_apply_ms = st["ntd_ms"] / max(st["napply"], 1)
    algo_bytes = NTD_BYTES[args.precision] * n
    achieved = algo_bytes / (ntd_per_apply_ms * 1e-3) / 1e9 if ntd_per_apply_ms > 0 else None
    depth = (grid[2] + 1) * (grid[1] + 1)  # dependent line solves per apply
    spmv_per_ms = st["spmv_ms"] / max(st["iters"], 1)
    spmv_achieved = SPMV_BYTES * n / (spmv_per_ms * 1e-3) / 1e9 if spmv_per_ms > 0 else None
    spmv_ops = SPMV_FP64_OPS * n / (spmv_per_ms * 1e-3) / 1e9 if spmv_per_ms > 0 else None
    reasons = sorted(set(clocks.get("reasons", [])) | set((fp64 or {}).get("clocks", {}).get("reasons", [])))
    clocks = dict(clocks, reasons=reasons)
    filt = ("rowsum" if net is None else
            "learned (conv net on log10 kappa, inference inside the step, weights "
            + os.path.basename(args.weights) + ")")
    line = {
        "metric": METRIC,
        "value": ms / 1e3 / ws,          # seconds per solve for the whole job (N replicas in parallel)
        "unit": "s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64+f32" if args.precision != "fp64" else "f64",
        "data": "synthetic",
        "config": {
            "workload": args.workload + ": " + describe(args.workload),
            "precond": {"combo": "B_c = NTD + ILU(0) (Sec. III Eq. (com))",
                        "ntd": "B_NTD (Sec. II)"}[args.precond],
            "factors": args.precision,
            "schur": {"newton": "X = 2 beta - beta P beta (Sec. II-A as printed)",
                      "beta": "X = beta (classical filtering; FFP_SCHUR_BETA)"}[args.schur],
            "filter": filt,
            "rtol": args.rtol,
            "setup_ms": setup_ms,
            "solve_ms": ms - setup_ms,
            "iters": st["iters"],
            "iters_rec": st["iters_rec"],
            "rel_res_true": st["rel_res_true"],
            "cond_est": st["cond_est"],
            "converged": ok,
            "fp64_rowsum": fp64,
            "speedup_vs_fp64_rowsum": (fp64["s"] / (ms / 1e3)) if fp64 else None,
            "replicas": ws,
            "l2": (f"inputs larger than L2 (each FP64 vector {8 * n / 1e6:.0f} MB > 129 MB)" if 8 * n > L2_BYTES
                   else f"working set larger than L2 (workspace {wsb / 1e6:.0f} MB > 129 MB, each FP64 "
                        f"vector {8 * n / 1e6:.0f} MB)" if wsb > L2_BYTES else
                   f"fits in L2 (workspace {wsb / 1e6:.0f} MB): not a bench-grade timing"),
        },
        "roofline": {
            "kernel": "apply_kernel (B_NTD sweeps, 3 launches per apply)",
            "bound": "hbm",
            "achieved": achieved,
            "peak": peak,
            "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None,
            "peak_kind": peak_kind,
            "traffic": APPLY_TRAFFIC.get((args.workload, args.precision)),
            "bytes_per_unknown": NTD_BYTES[args.precision],
            "algorithmic_bytes_per_apply": algo_bytes,
            "ms_per_apply": ntd_per_apply_ms,
            "governing_bound": "dependency chain, not bandwidth: (nz+1)(ny+1) dependent line solves "
                               "per apply; the time per line solve sets the apply's time",
            "dependent_line_solves_per_apply": depth,
            "ns_per_line_solve": ntd_per_apply_ms * 1e6 / depth,
        },
        "roofline_spmv": {
            "kernel": "spmv_dot_kernel (q = A p fused with (p, q))",
            "bound": "alu",
            "achieved": spmv_ops,
            "peak": FP64_OPS_PEAK / 1e9,
            "unit": "G FP64 FMA-pipe ops/s",
            "frac": (spmv_ops * 1e9 / FP64_OPS_PEAK) if spmv_ops else None,
            "peak_kind": "derived: 152 SMs x 2 FP64 FMA/clock x 2070 MHz (nominal 1.25 TFLOP/s FP64)",
            "ops_per_unknown": SPMV_FP64_OPS,
            "hbm_achieved_gbs": spmv_achieved,
            "hbm_frac": (spmv_achieved / peak) if spmv_achieved else None,
            "hbm_peak_kind": peak_kind,
            "traffic": SPMV_TRAFFIC.get(args.workload),
            "bytes_per_unknown": SPMV_BYTES,
            "ms_per_launch": spmv_per_ms,
        },
        "e2e": {"value": e2e_ms / 1e3 / ws, "unit": "s", "steps": e2e_steps,
                "h2d_bytes_per_step": 2 * 8 * n, "d2h_bytes_per_step": 8 * n},
        "gpu_launches": int(sum(s["launches"] for s in stats))
        + args.steps * (ffp.setup_launches(grid, args.precond, user_t=net is not None)
                        + (6 if net is not None else 0)),
        "clocks": clocks,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, args.workload, st["iters"], args.cpu_sample_iters)
    if ws > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


def run_batched(args):
    """The batched workload: every step sets up all 64 instances and solves
    all 256 (instance, right-hand side) pairs to rtol in one batch, launch
    configuration from the autotuner (tuned once, in the first warm-up step).
    On N ranks the job is one list of 64 N instances (weak scaling), split by
    lpt_partition on n; each rank sets up and solves its share as one batch,
    with no collective on the data path."""
    import torch
    import torch.distributed as dist
    from paper_1909_09771_gb300 import ffp
    from paper_1909_09771_gb300 import inputs as I

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nrhs = 4
    count = 64 * ws
    all_grids = I.batched_grids(seed=args.seed, count=count)
    mine = lpt_partition([int(np.prod(g)) for g in all_grids], ws)[rank]
    insts = I.workload_batched(seed=args.seed, count=count, nrhs=nrhs, indices=mine)
    grids = [w["grid"] for w in insts]
    bcs = [w["bc"] for w in insts]
    ns = [int(np.prod(g)) for g in grids]
    kap_h = [torch.from_numpy(w["kappa"]).pin_memory() for w in insts]
    b_h = [torch.from_numpy(np.ascontiguousarray(b)).pin_memory() for w in insts for b in w["b"]]
    x_h = [torch.empty(ns[p // nrhs], dtype=torch.float64).pin_memory() for p in range(len(b_h))]
    kap = [k.to(dev) for k in kap_h]
    bs = [b.to(dev) for b in b_h]
    xs = [torch.zeros_like(b) for b in bs]
    stream = torch.cuda.current_stream(dev)
    wsb = ffp.batch_workspace_bytes(grids, nrhs, args.precision)
    work = torch.empty(wsb, dtype=torch.uint8, device=dev)
    tuned = {}

    def step(kaps, rhs, xout):
        bat = ffp.Batch(grids, kaps, bcs, nrhs=nrhs, precision=args.precision,
                        precond=args.precond, workspace=work)
        if not tuned:
            tuned.update(bat.tune())
        else:
            bat.set_config(tuned["ilu_warps"], tuned["branches"], tuned["rhs_per_cta"])
        for x in xout:
            x.zero_()
        _, stats = bat.solve(rhs, xs=xout, rtol=RTOL, maxit=MAXIT, check=False)
        info = bat.info()
        bat.close()
        return stats, info

    def barrier():
        if ws > 1:
            dist.barrier()

    for _ in range(args.warmup):
        stats, info = step(kap, bs, xs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    runs = []
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            runs.append(step(kap, bs, xs))
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    e2 = []
    barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        kd = [k.to(dev, non_blocking=True) for k in kap_h]
        bd = [b.to(dev, non_blocking=True) for b in b_h]
        step(kd, bd, xs)
        for xh, xd in zip(x_h, xs):
            xh.copy_(xd, non_blocking=True)
        t1.record(stream)
        torch.cuda.synchronize()
        e2.append(t0.elapsed_time(t1))
    barrier()
    e2e_ms = sum(e2) / len(e2)
    ms, e2e_ms = max_over_ranks([ms, e2e_ms], dev, ws)
    stats, info = runs[-1]
    ok = all(s["status"] == 0 and s["rel_res_true"] < RTOL for st, _ in runs for s in st)
    ok = bool(max_over_ranks([0.0 if ok else 1.0], dev, ws)[0] == 0.0)
    stats = merge_pair_stats(stats, mine, nrhs, count, ws)
    iters = [s["iters"] for s in stats]
    sizes = [int(np.prod(g)) for g in all_grids]
    loads = [sum(sizes[i] for i in part) for part in lpt_partition(sizes, ws)]
    peak, peak_kind = load_peaks()
    pair_unknowns = sum(ns[p // nrhs] for p in range(len(bs)))   # this rank's
    job_pair_unknowns = nrhs * sum(sizes)
    algo_bytes = NTD_BYTES[args.precision] * pair_unknowns
    ntd_ms = tuned.get("ntd_ms", 0.0)
    achieved = algo_bytes / (ntd_ms * 1e-3) / 1e9 if ntd_ms > 0 else None
    line = {
        "metric": METRIC,
        "value": ms / 1e3 / ws,
        "unit": "s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64+f32" if args.precision != "fp64" else "f64",
        "data": "synthetic",
        "config": {
            "workload": "batched: " + describe("batched"),
            "precond": {"combo": "B_c = NTD + ILU(0) (Sec. III Eq. (com))",
                        "ntd": "B_NTD (Sec. II)"}[args.precond],
            "factors": args.precision,
            "filter": "rowsum",
            "rtol": RTOL,
            "unknowns": sum(sizes),
            "pairs": len(stats),
            "pair_unknowns_per_s": job_pair_unknowns / (ms / 1e3),
            "sharding": (f"LPT on n = nx ny nz over {ws} ranks: {count} instances, loads "
                         f"max/mean {max(loads) / (sum(loads) / ws):.3f}") if ws > 1 else "one rank",
            "iters_mean": float(np.mean(iters)),
            "iters_max": int(max(iters)),
            "converged": ok,
            "tuned": tuned,
            "groups": info["groups"],
            "replicas": ws,
            "l2": "inputs larger than L2 (the batch's vectors total several GB)",
        },
        "roofline": {
            "kernel": "apply_kernel (B_NTD sweeps of all 256 pairs, 3 launches per slot-count group)",
            "bound": "hbm",
            "achieved": achieved,
            "peak": peak,
            "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None,
            "peak_kind": peak_kind,
            "traffic": None,
            "algorithmic_bytes_per_apply": algo_bytes,
            "ms_per_apply": ntd_ms,
        },
        "e2e": {"value": e2e_ms / 1e3 / ws, "unit": "s",
                "h2d_bytes_per_step": 8 * (sum(sizes) + job_pair_unknowns),
                "d2h_bytes_per_step": 8 * job_pair_unknowns},
        "gpu_launches": int(max_over_ranks([sum(st[0]["launches"] + inf["setup_launches"]
                                                for st, inf in runs)], dev, ws)[0]) * ws,
        "clocks": clk.summary(),
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_batched(insts, iters, nrhs)
    if ws > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


def cpu_baseline_batched(insts, iters, nrhs):
    """The oracle on a bounded sample of the batch: instance 0's assembly +
    setup + ILU(0) pivots and one B_c flexible-CG iteration, measured, then
    scaled by unknowns to every instance's setup and every pair's iterations."""
    from oracle import oracle as O
    w = insts[0]
    g = w["grid"]
    n0 = int(np.prod(g))
    t0 = time.perf_counter()
    bands = O.assemble(g, w["kappa"], w["bc"])
    f = O.setup(g, bands)
    D = O.ilu0_setup(g, bands)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    O.pcg(g, bands, f, w["b"][0], rtol=1e-300, maxit=1, flexible=True, ilu=D)
    t_iter = time.perf_counter() - t0
    ns = [int(np.prod(x["grid"])) for x in insts]
    total = t_setup / n0 * sum(ns) + t_iter / n0 * sum(iters[p] * ns[p // nrhs] for p in range(len(iters)))
    return {"value": total, "unit": "s", "cores": 1, "kind": "oracle",
            "sample": f"instance 0 ({g[0]}x{g[1]}x{g[2]}): setup {t_setup:.2f} s and one B_c "
                      f"flexible-CG iteration {t_iter:.2f} s measured, scaled by unknowns to all "
                      f"{len(insts)} setups and {len(iters)} solves ({sum(iters)} iterations)"}


def oracle_iterations(workload):
    """The oracle's own iteration count for a workload (B_c, FP64, rowsum,
    rtol 1e-8), stored by oracle/reference_iterations.py, or None."""
    p = os.path.join(ROOT, "oracle", "reference_iterations.json")
    try:
        with open(p) as fh:
            return json.load(fh)[workload]["iters"]
    except Exception:
        return None


def cpu_baseline(w, workload, gpu_iters, sample_iters):
    """The oracle as it stands, one host core: assembly + setup + ILU(0) pivots
    measured in full, plus `sample_iters` flexible-CG iterations with B_c
    measured; the solve is extrapolated to the oracle's own iteration count
    for this workload (stored by oracle/reference_iterations.py), or to the
    GPU's count where none is stored.  Returns the line's cpu_baseline object."""
    from oracle import oracle as O
    g = w["grid"]
    t0 = time.perf_counter()
    bands = O.assemble(g, w["kappa"], w["bc"])
    f = O.setup(g, bands)
    D = O.ilu0_setup(g, bands)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    O.pcg(g, bands, f, w["b"], rtol=1e-300, maxit=sample_iters, flexible=True, ilu=D)
    t_iter = (time.perf_counter() - t0) / sample_iters
    iters = oracle_iterations(workload)
    src = "the oracle's own count, oracle/reference_iterations.json"
    if iters is None:
        iters, src = gpu_iters, "the GPU solve's count (no oracle count stored for this workload)"
    return {"value": t_setup + iters * t_iter, "unit": "s", "cores": 1, "kind": "oracle",
            "extrapolated": True,
            "sample": f"EXTRAPOLATED: setup measured in full ({t_setup:.1f} s) + {sample_iters} B_c "
                      f"flexible-CG iterations measured ({t_iter:.2f} s each), times {iters} iterations "
                      f"({src}); rowsum filter, FP64"}


def run_reference(args):
    """CPU oracle on a bounded sample per step (rank 0 only)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    iters = oracle_iterations(args.workload)
    if args.workload == "batched":
        from paper_1909_09771_gb300 import inputs as I
        insts = I.workload_batched(seed=args.seed)
        per_pair = [iters if iters else 1] * (4 * len(insts))
    else:
        w = make_workload(args.workload, seed=args.seed)
    times = []
    for k in range(args.warmup + args.steps):
        if args.workload == "batched":
            cb = cpu_baseline_batched(insts, per_pair, 4)
        else:
            cb = cpu_baseline(w, args.workload, 1, 1)
        if k >= args.warmup:
            times.append(cb["value"])
    v = sum(times) / len(times)
    line = {"metric": METRIC, "value": v, "unit": "s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.workload + ": " + describe(args.workload),
                       "precond": "B_c = NTD + ILU(0) (Sec. III Eq. (com))", "rtol": RTOL},
            "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# DRAM bytes per launch from one ncu capture of the current kernels (dram__bytes_read.sum +
# dram__bytes_write.sum), by workload (and factor precision); absent = not measured for the
# kernel as it now is.
APPLY_TRAFFIC = {("grf350", "fp32"): 2676.0e6}   # the three sweep launches of one apply
SPMV_TRAFFIC = {"grf350": 2657.7e6}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="grf350")
    ap.add_argument("--rtol", type=float, default=RTOL)
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "bf16"])
    ap.add_argument("--precond", default="combo", choices=["combo", "ntd"])
    ap.add_argument("--schur", default="newton", choices=["newton", "beta"],
                    help="approximate inverse in the Schur terms: newton = 2 beta - beta P beta "
                         "(Sec. II-A as printed), beta = the classical X = beta")
    ap.add_argument("--filter", default="learned", choices=["rowsum", "learned"])
    ap.add_argument("--weights", default=os.path.join(ROOT, "paper_1909_09771_gb300",
                                                        "learned_filter_weights.txt"))
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-sample-iters", type=int, default=2)
    ap.add_argument("--fp64-steps", type=int, default=1,
                    help="timed solves of the plain FP64 rowsum form beside the main arm (0: none)")
    ap.add_argument("--e2e-steps", type=int, default=3, help="end-to-end steps (at least 1)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
