"""The paper's own test problems (Sec. IV, "Test Matrices"; Table I) on the GPU.

  parity     at 24^3, each matrix type: B_c flexible CG with FP64 factors against
             the FP64 oracle, to 1e-10 -- iterations equal +-1, solutions within
             1e-7 relative, both converged (the PCG bar of the other parity tests)
  Table I    at 100^3 (the smallest size Table I lists), FP32 factors, tol 1e-7
             and 1e-10: the iteration at which the recursive residual meets tol,
             printed next to the paper's count.  Asserted: every solve meets
             1e-7 on the true residual and reaches 1e-10 on the recursive one;
             on the Poisson matrix (type 3) the count is within 1.5x of Table I.
             Types 1 and 2 need more iterations here than Table I reports; the
             right-hand side and the treatment of the jumps are not stated in the
             paper, see the design notes.
"""
import os

import numpy as np
import pytest
import torch

from oracle import oracle as o
from paper_1909_09771_gb300 import build as B
from paper_1909_09771_gb300 import ffp
from paper_1909_09771_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_table1.txt")


def load_table1():
    """(type, n, tol) -> Table I iteration count."""
    rows = {}
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            kind, n, tol, _, _, _, iters = line.split()
            rows[(int(kind), int(n), float(tol))] = {"iters": int(iters)}
    return rows


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    ffp.load()


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("kind", [1, 2, 3])
def test_paper_problem_parity_fp64(kind):
    w = I.workload_paper(kind, 24)
    g, bc = w["grid"], w["bc"]
    P = ffp.Preconditioner(g, dev(w["kappa"]), bc, "fp64", precond="combo")
    x, st = P.solve(dev(w["b"]), rtol=1e-10, maxit=400)
    bands = o.assemble(g, w["kappa"], bc)
    ref = o.pcg(g, bands, o.setup(g, bands), w["b"], rtol=1e-10, maxit=400, flexible=True,
                ilu=o.ilu0_setup(g, bands))
    assert st["status"] == 0 and ref["status"] == 0 and st["rel_res_true"] < 1e-10
    assert abs(st["iters"] - ref["iters"]) <= 1, (st["iters"], ref["iters"])
    assert relerr(x.cpu().numpy(), ref["x"]) <= 1e-7


@pytest.mark.parametrize("kind", [1, 2, 3])
def test_table1_iterations_100(kind):
    table = load_table1()
    w = I.workload_paper(kind, 100)
    P = ffp.Preconditioner(w["grid"], dev(w["kappa"]), w["bc"], "fp32", precond="combo")
    b = dev(w["b"])
    for tol in (1e-7, 1e-10):
        _, st = P.solve(b, rtol=tol, maxit=300, check=False)
        paper = table[(kind, 100, tol)]["iters"]
        print(f"type {kind}, 100^3, tol {tol:g}: {st['iters_rec']} iterations "
              f"(true residual {st['rel_res_true']:.2e} after {st['iters']}); Table I: {paper}")
        assert st["iters_rec"] > 0
        if tol == 1e-7:
            assert st["status"] == 0 and st["rel_res_true"] < tol
        if kind == 3:
            assert st["iters_rec"] <= 1.5 * paper
