"""Cycle budget of the apply's line steps (FP32 factors), from the profiling
build of the library (python -m paper_1909_09771_gb300.build --profile, which
writes libffp_profile.so beside libffp.so; the normal library has no stamps).

It also reports the setup (slot counts 8 and 11, so nx from 130 to 353): its
time (CUDA events), and per plane step of the first level-3 half the chain
CTA's phases, the level-2 factorization of the plane (line Schur terms, line
pivots, line stores) and the nested plane solve for beta-hat; the cell-wise
phases (beta-hat, the next plane's Schur term) run as a separate launch over
the whole GPU.

The profiling build stamps clock64 around the segments of every line step of
one compute warp (level-2 half 0 of the first level-3 half, phase 0 launch)
and reports, per lower- and upper-sweep step: the wait for its shared-memory
stage, the right-hand side (loads and coupling terms), the line solve (loads
of the line's multipliers and the twisted solve), and the store plus stage
release.  The stamps themselves cost some cycles, so the total is a little
above the uninstrumented step (compare ns_per_line_solve of bench.py).

  python -m paper_1909_09771_gb300.profile_steps [n ...]    (grf<n> workloads, default 350)
"""
from __future__ import annotations

import ctypes
import os
import sys

import torch

from paper_1909_09771_gb300 import ffp
from paper_1909_09771_gb300 import inputs as I


def budget(n, lib):
    w = I.workload_grf(seed=0, n=n)
    kap = torch.as_tensor(w["kappa"], device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    P = ffp.Preconditioner(w["grid"], kap, w["bc"], "fp32")
    e1.record()
    torch.cuda.synchronize()
    setup_ms = e0.elapsed_time(e1)
    _, st = P.solve(torch.as_tensor(w["b"], device="cuda"), rtol=1e-30, maxit=5, check=False)
    torch.cuda.synchronize()
    prof = (ctypes.c_ulonglong * 16)()
    if lib.ffp_step_profile(ctypes.cast(prof, ctypes.c_void_p)) != 0:
        raise RuntimeError("ffp_step_profile failed")
    p = list(prof)
    sprof = (ctypes.c_ulonglong * 16)()
    setup = None
    if lib.ffp_setup_profile(ctypes.cast(sprof, ctypes.c_void_p)) == 0 and sprof[8] > 0:
        q = list(sprof)
        npl = q[8]
        # the chain CTAs' phases per plane step; the cell-wise phases run as a separate
        # launch over the whole GPU and are in setup_ms only
        setup = {"planes": npl, "level2": q[0] / npl, "line_schur": q[5] / npl, "line_pivots": q[6] / npl,
                 "line_store": q[7] / npl, "plane_solve": q[2] / npl, "setup_ms": setup_ms}
    depth = (w["grid"][2] + 1) * (w["grid"][1] + 1)
    ms = st["ntd_ms"] / max(st["napply"], 1)
    nl, nu = max(p[4], 1), max(p[9], 1)
    P.close()
    return {
        "grid": w["grid"], "ms_per_apply": ms, "ns_per_line_step": ms * 1e6 / depth,
        "lower": {"steps": p[4], "wait": p[0] / nl, "rhs": p[1] / nl, "solve": p[2] / nl,
                  "store_release": p[3] / nl, "total": sum(p[0:4]) / nl},
        "upper": {"steps": p[9], "wait": p[5] / nu, "rhs": p[6] / nu, "solve": p[7] / nu,
                  "store_release": p[8] / nu, "total": sum(p[5:9]) / nu},
        "loop_cycles_per_step": p[10] / max(p[4] + p[9], 1),
        "first_try_misses": p[11],
        "setup": setup,
    }


def main(argv):
    from paper_1909_09771_gb300 import build as B
    ffp.LIB_PATH = B.build(profile=True)
    lib = ffp.load()
    lib.ffp_step_profile.argtypes = [ctypes.c_void_p]
    lib.ffp_step_profile.restype = ctypes.c_int
    lib.ffp_setup_profile.argtypes = [ctypes.c_void_p]
    lib.ffp_setup_profile.restype = ctypes.c_int
    for n in ([int(a) for a in argv] or [350]):
        r = budget(n, lib)
        print(f"grf{n} {r['grid']}: {r['ms_per_apply']:.2f} ms per apply, "
              f"{r['ns_per_line_step']:.0f} ns per line step (profiling build)")
        for k in ("lower", "upper"):
            q = r[k]
            print(f"  {k} steps {q['steps']}: wait {q['wait']:.0f}  rhs {q['rhs']:.0f}  solve "
                  f"{q['solve']:.0f}  store+release {q['store_release']:.0f}  total {q['total']:.0f} cycles")
        print(f"  plane loop {r['loop_cycles_per_step']:.0f} cycles per step; stage waits whose first "
              f"try failed: {r['first_try_misses']}")
        q = r["setup"]
        if q:
            print(f"  setup {q['setup_ms']:.0f} ms (profiling build, CUDA events); chain-CTA cycles per "
                  f"plane step ({q['planes']} steps of one level-3 half): level-2 {q['level2']:.0f} (line "
                  f"Schur {q['line_schur']:.0f}, pivots {q['line_pivots']:.0f}, stores {q['line_store']:.0f}), "
                  f"plane solve {q['plane_solve']:.0f}")


if __name__ == "__main__":
    main(sys.argv[1:])
