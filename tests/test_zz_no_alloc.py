"""The allocation-free apply, ffp_apply_noalloc, against ffp_apply.

ffp_apply_noalloc serves callers that cannot allocate device memory when they
apply the preconditioner (code running under a framework that owns every
device allocation, or steady-state code that must never call cudaMalloc): it
keeps its two scratch planes in a fixed array inside the library instead of
the caller's workspace.  Its results must equal those of ffp_apply, which
runs the same kernels with workspace scratch.  This file is collected last so
that a run stopping at the first failure has already run every other test;
it passes alone and after the others.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1909_09771_gb300 import build as B
from paper_1909_09771_gb300 import ffp
from paper_1909_09771_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    lib = ffp.load()
    lib.ffp_apply_noalloc.argtypes = [ctypes.c_void_p] * 4
    lib.ffp_apply_noalloc.restype = ctypes.c_int
    return lib


def _noalloc(lib, P, r):
    z = torch.full_like(r, float("nan"))
    st = lib.ffp_apply_noalloc(P._h, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, z


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_apply_matches_apply_on_two_calls(lib, precision):
    grid = (45, 37, 13)
    w = I.random_small(grid, 41, contrast_exp=3)
    P = ffp.Preconditioner(grid, torch.as_tensor(w["kappa"], device="cuda"), w["bc"], precision)
    n = int(np.prod(grid))
    for seed in (1, 2):     # two calls in a row, different right-hand sides
        r = torch.as_tensor(np.random.default_rng(seed).standard_normal(n), device="cuda")
        z_ref = P.apply(r)
        st, z = _noalloc(lib, P, r)
        assert st == ffp.FFP_OK
        err = float(torch.linalg.norm(z - z_ref) / torch.linalg.norm(z_ref))
        assert err <= 1e-12, err
    P.close()


def test_noalloc_rejects_planes_beyond_the_fixed_scratch(lib):
    grid = (400, 400, 1)    # 160000 cells per plane > FFP_NOALLOC_MAX_PLANE
    assert grid[0] * grid[1] > 131072
    P = ffp.Preconditioner(grid, torch.ones(grid[0] * grid[1], dtype=torch.float64, device="cuda"),
                           I.BC_Z_DIRICHLET, "fp32")
    r = torch.ones(grid[0] * grid[1], dtype=torch.float64, device="cuda")
    st, _ = _noalloc(lib, P, r)
    assert st == ffp.FFP_ERR_ARG
    P.close()


@pytest.mark.parametrize("ny, ok", [(800, True), (1000, False)])
def test_noalloc_line_block_size_rule(lib, ny, ok):
    """nx = 3 with FP64 factors: S = 1 slot per lane, padded to SP = 4, so one
    scratch plane in the line-block layout holds ny * (32 * 4 + 32) = 160 ny
    FP64 values.  The plane has only 3 ny cells (far below the cell limit), so
    ny = 1000 (1.28 MB > 1 MiB) is rejected by the line-block rule alone, while
    ny = 800 (1.024 MB) fits and gives ffp_apply's result."""
    grid = (3, ny, 2)
    assert grid[0] * grid[1] <= 131072
    assert (ny * 160 * 8 <= 8 * 131072) == ok
    w = I.random_small(grid, 43, contrast_exp=3)
    P = ffp.Preconditioner(grid, torch.as_tensor(w["kappa"], device="cuda"), w["bc"], "fp64")
    r = torch.as_tensor(np.random.default_rng(3).standard_normal(int(np.prod(grid))), device="cuda")
    st, z = _noalloc(lib, P, r)
    if ok:
        assert st == ffp.FFP_OK
        z_ref = P.apply(r)
        assert float(torch.linalg.norm(z - z_ref) / torch.linalg.norm(z_ref)) <= 1e-12
    else:
        assert st == ffp.FFP_ERR_ARG
    P.close()
