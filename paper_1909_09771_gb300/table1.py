"""The paper's Table I experiment with this library: the three test matrices of
Sec. IV (type 1 skyscrapers, type 2 ring, type 3 Poisson; unit cube, Dirichlet
on all faces, b = h^3) at n = 100, 200, 350 and tolerances 1e-7, 1e-10, solved
with the combination preconditioner B_c (Sec. III Eq. (com)) by flexible CG
from x0 = 0, on one GPU.

Per row: the setup (assembly, NTD factorization, ILU(0) pivots) and the solve
timed with CUDA events on the current stream, the CG iterations, the first
iteration at which the recursive residual met the tolerance, and the true
relative residual.  One warm-up setup and solve of the smallest row come first.

  python -m paper_1909_09771_gb300.table1 [--sizes 100,200,350] [--tols 1e-7,1e-10]
        [--precision fp32] [--precond combo] [--schur newton] [--maxit 1000] [--json out.json]
"""
from __future__ import annotations

import argparse
import json
import sys

import torch

from paper_1909_09771_gb300 import ffp
from paper_1909_09771_gb300 import inputs as I


def run_row(kind, n, tol, precision, precond, schur, maxit):
    w = I.workload_paper(kind, n)
    dev = torch.device("cuda")
    kappa = torch.as_tensor(w["kappa"], device=dev)
    b = torch.as_tensor(w["b"], device=dev)
    st = torch.cuda.current_stream()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(st)
    P = ffp.Preconditioner(w["grid"], kappa, w["bc"], precision, precond=precond, schur=schur)
    e1.record(st)
    _, s = P.solve(b, rtol=tol, maxit=maxit, check=False)
    e2.record(st)
    torch.cuda.synchronize()
    P.close()
    return {"type": kind, "n": n, "tol": tol, "setup_s": e0.elapsed_time(e1) / 1e3,
            "solve_s": e1.elapsed_time(e2) / 1e3, "iters": s["iters"], "iters_rec": s["iters_rec"],
            "rel_res_true": s["rel_res_true"], "status": s["status"]}


def main(argv):
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", default="100,200,350")
    ap.add_argument("--tols", default="1e-7,1e-10")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "bf16"])
    ap.add_argument("--precond", default="combo", choices=["combo", "ntd"])
    ap.add_argument("--schur", default="newton", choices=["newton", "beta"])
    ap.add_argument("--maxit", type=int, default=1000)
    ap.add_argument("--json", default=None)
    args = ap.parse_args(argv)
    sizes = [int(v) for v in args.sizes.split(",")]
    tols = [float(v) for v in args.tols.split(",")]
    run_row(3, min(sizes), tols[0], args.precision, args.precond, args.schur, args.maxit)  # warm-up
    rows = []
    print(f"| type | n | tol | iterations | recursive residual met at | true residual | setup (s) | "
          f"solve (s) | status |  ({args.precision}, {args.precond}, schur {args.schur})")
    print("|---|---|---|---:|---:|---|---:|---:|---|")
    for tol in tols:
        for kind in (1, 2, 3):
            for n in sizes:
                r = run_row(kind, n, tol, args.precision, args.precond, args.schur, args.maxit)
                rows.append(r)
                print(f"| {kind} | {n} | {tol:g} | {r['iters']} | {r['iters_rec']} | {r['rel_res_true']:.1e} | "
                      f"{r['setup_s']:.2f} | {r['solve_s']:.2f} | {r['status']} |", flush=True)
    if args.json:
        with open(args.json, "w") as fh:
            json.dump({"args": vars(args), "rows": rows}, fh, indent=1)


if __name__ == "__main__":
    main(sys.argv[1:])
