"""Iteration counts of the CPU oracle's own solves, stored for the benchmark.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): bench.py's CPU-baseline
and reference legs extrapolate the oracle's time per iteration to the number of
iterations the oracle itself needs, and that number comes from here, never from
the CUDA library.  The script calls only the oracle and the seeded input
generators; it writes oracle/reference_iterations.json.

Each entry is one full oracle solve: FP64 factors, rowsum filter, the
combination preconditioner B_c (Sec. III Eq. (com)), flexible CG from x0 = 0 to
||b - A x|| / ||b|| < 1e-8 (Sec. III conventions, the true residual confirmed).
The batched workload is sampled: its first `--batched-instances` instances
with all their right-hand sides.

  python -m oracle.reference_iterations [--workloads grf350,blocks32,batched]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(_HERE))

from oracle import oracle as O  # noqa: E402
from paper_1909_09771_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(_HERE, "reference_iterations.json")
RTOL = 1e-8
MAXIT = 1000


def solve_count(w, b):
    g = w["grid"]
    t0 = time.perf_counter()
    bands = O.assemble(g, w["kappa"], w["bc"])
    f = O.setup(g, bands)
    D = O.ilu0_setup(g, bands)
    res = O.pcg(g, bands, f, b, rtol=RTOL, maxit=MAXIT, flexible=True, ilu=D)
    return int(res["iters"]), int(res["status"]), float(res["relres"]), time.perf_counter() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workloads", default="grf350,blocks32,batched")
    ap.add_argument("--batched-instances", type=int, default=2)
    args = ap.parse_args()
    out = {}
    if os.path.exists(OUT):
        with open(OUT) as fh:
            out = json.load(fh)
    for name in args.workloads.split(","):
        if name == "batched":
            insts = I.workload_batched(seed=0)[: args.batched_instances]
            its = []
            for w in insts:
                for b in w["b"]:
                    k, st, rr, _ = solve_count(w, np.ascontiguousarray(b))
                    assert st == 0, (w["grid"], st)
                    its.append(k)
            out[name] = {"iters": float(np.mean(its)), "per_pair": its,
                         "sample": f"first {len(insts)} instances x {len(insts[0]['b'])} "
                                   f"right-hand sides (seed 0)"}
        else:
            w = {"grf350": lambda: I.workload_grf(seed=0, n=350),
                 "blocks32": lambda: I.workload_blocks32(seed=0),
                 "layered128": lambda: I.workload_layered128(seed=0)}[name]()
            k, st, rr, sec = solve_count(w, w["b"])
            out[name] = {"iters": k, "status": st, "rel_res_true": rr, "oracle_s": round(sec, 1)}
        print(name, out[name], flush=True)
        with open(OUT, "w") as fh:
            json.dump(out, fh, indent=1, sort_keys=True)
            fh.write("\n")


if __name__ == "__main__":
    main()
