"""The failure path of the bounded waits, exercised without faulting the GPU.

Every wait inside the apply kernels has a try limit; a wait that runs out
records a timeout flag and lets the kernel run to its end, and the CG driver
then returns FFP_ERR_TIMEOUT.  The test hook ffp_debug_stall makes one
producer warp withhold its first "stage full" signal (a flag that nothing
else sets), with a short try limit, and checks that:
  * the solve returns FFP_ERR_TIMEOUT after its first iteration (not a hang,
    not a fault);
  * the context stays usable: with the hook off, the same handle solves the
    same problem to the same iterate as a fresh handle.
"""
import numpy as np
import pytest
import torch

from paper_1909_09771_gb300 import build as B
from paper_1909_09771_gb300 import ffp
from paper_1909_09771_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    ffp.load()


@pytest.mark.parametrize("precision, precond", [("fp32", "ntd"), ("fp64", "combo")])
def test_withheld_signal_times_out_and_recovers(precision, precond):
    grid = (40, 12, 10)
    w = I.random_small(grid, 51, contrast_exp=2)
    kappa = torch.as_tensor(w["kappa"], device="cuda")
    b = torch.as_tensor(w["b"], device="cuda")
    P = ffp.Preconditioner(grid, kappa, w["bc"], precision, precond=precond)
    P.debug_stall(1, wait_tries=2048)
    _, st = P.solve(b, rtol=1e-8, maxit=50, check=False)
    torch.cuda.synchronize()
    assert st["status"] == ffp.FFP_ERR_TIMEOUT, st
    assert st["iters"] == 1
    P.debug_stall(0)
    x1, st1 = P.solve(b, rtol=1e-8, maxit=500)
    Q = ffp.Preconditioner(grid, kappa, w["bc"], precision, precond=precond)
    x2, st2 = Q.solve(b, rtol=1e-8, maxit=500)
    assert st1["status"] == 0 and st1["iters"] == st2["iters"]
    assert torch.equal(x1, x2)
    P.close()
    Q.close()


def test_debug_stall_rejects_unknown_mode():
    grid = (8, 4, 4)
    P = ffp.Preconditioner(grid, torch.ones(128, dtype=torch.float64, device="cuda"), I.BC_Z_DIRICHLET)
    with pytest.raises(ffp.FFPError) as e:
        P.debug_stall(7)
    assert e.value.status == ffp.FFP_ERR_ARG
    P.close()
