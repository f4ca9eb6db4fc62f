"""GPU parity at the sizes the bench runs.

  grf350      the 350^3 Gaussian-random-field workload (42.875M unknowns,
              contrast 10^6): one setup and one B_NTD apply, FP64 and FP32
              factors, compared with the oracle entry by entry;
  grf128,     the same field at 128^3 and the 128^3 layered workload (layers
  layered128  1 / 1e6 with inclusions of 1e-3): one flexible-CG solve with the
              combination preconditioner B_c (Sec. III Eq. (com)), FP64 factors.

Tolerances are those of tests/test_gpu_parity.py, derived at run time by
tests/parity_bounds.py: per entry in units of s = B^{-1}|r| (B^{-1} is
entrywise non-negative), so that an error confined to one twist plane, one
line or the tail lanes cannot hide in a norm over 42.9M entries.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as o
from paper_1909_09771_gb300 import build as B
from paper_1909_09771_gb300 import ffp
from paper_1909_09771_gb300 import inputs as I
from tests import parity_bounds as PB

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    ffp.load()


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


class Ref:
    """The oracle's side of the 350^3 comparison, computed once."""


@pytest.fixture(scope="module")
def grf350():
    w = I.workload_grf(seed=0, n=350)
    R = Ref()
    R.w = w
    R.grid = w["grid"]
    R.bands = o.assemble(R.grid, w["kappa"], w["bc"])
    R.f = o.setup(R.grid, R.bands)
    R.r = np.random.default_rng(350).standard_normal(int(np.prod(R.grid)))
    R.s, R.z = PB.apply_scale(R.f, R.r)
    R.kf, R.amp = PB.sensitivity(R.grid, R.bands, R.f, R.r, R.s)
    return R


def gpu_factors(P):
    ex = {k: host(v) for k, v in P.export(("l3", "l2", "l1", "minv")).items()}
    nan = np.full(ex["l3"].size, np.nan)
    return o.Factors(P.grid, ex["l3"], nan, nan, ex["l2"], nan, ex["l1"], 1.0 / ex["minv"]), ex


def test_grf350_fp64_setup_and_apply(grf350):
    R = grf350
    P = ffp.Preconditioner(R.grid, dev(R.w["kappa"]), R.w["bc"], "fp64")
    z = host(P.apply(dev(R.r)))
    fg, ex = gpu_factors(P)
    P.close()
    del P
    # the stored factors, per entry
    tol = PB.factor_tol(R.grid, R.kf)
    for k, ref in (("l2", R.f.Py), ("l1", R.f.To), ("minv", 1.0 / R.f.M)):
        err = float(np.max(np.abs(ex[k] - ref) / (np.abs(ref) + 1e-300)))
        assert err <= tol, (k, err, tol)
    del ex
    # the apply kernel on the GPU's own factors: 1e-12 per entry
    sg, zg = PB.apply_scale(fg, R.r)
    ok, worst = PB.per_entry_ok(z, zg, sg, 1e-12)
    assert ok, ("apply on the GPU's factors", worst)
    assert relerr(z, zg) <= 1e-12
    # setup + apply end to end against the oracle's own factors
    ok, worst = PB.per_entry_ok(z, R.z, R.s, PB.e2e_tol(R.grid, R.amp))
    assert ok, ("setup + apply", worst, PB.e2e_tol(R.grid, R.amp))


def test_grf350_fp32_apply(grf350):
    """FP32 factors and FP32 sweeps: against the oracle applying the exported
    FP32 factors (only the sweeps' FP32 arithmetic differs) per entry, and
    against the FP64 oracle with its own factors in the 2-norm (1e-5)."""
    R = grf350
    P = ffp.Preconditioner(R.grid, dev(R.w["kappa"]), R.w["bc"], "fp32")
    z = host(P.apply(dev(R.r)))
    fg, _ = gpu_factors(P)
    P.close()
    del P
    sg, zg = PB.apply_scale(fg, R.r)
    ok, worst = PB.per_entry_ok(z, zg, sg, 1e-5)
    assert ok, ("FP32 sweeps on FP32 factors", worst)
    assert relerr(z, R.z) <= 1e-5


def _combo_pcg_parity(w, rtol, xtol):
    g, bc = w["grid"], w["bc"]
    P = ffp.Preconditioner(g, dev(w["kappa"]), bc, "fp64", precond="combo")
    x, st = P.solve(dev(w["b"]), rtol=rtol, maxit=1000, check=False)
    xg = host(x)
    P.close()
    bands = o.assemble(g, w["kappa"], bc)
    ref = o.pcg(g, bands, o.setup(g, bands), w["b"], rtol=rtol, maxit=1000, flexible=True,
                ilu=o.ilu0_setup(g, bands))
    assert st["status"] == 0 and ref["status"] == 0, (st, ref["status"])
    assert abs(st["iters"] - ref["iters"]) <= 1, (st["iters"], ref["iters"])
    bn = np.linalg.norm(w["b"])
    # both true residuals, the GPU's recomputed with the oracle's operator
    assert st["rel_res_true"] < rtol and ref["relres"] < rtol
    assert np.linalg.norm(w["b"] - o.spmv(g, bands, xg)) / bn < rtol
    assert relerr(xg, ref["x"]) <= xtol, relerr(xg, ref["x"])
    return st["iters"], ref["iters"]


def test_grf128_combo_pcg_fp64():
    """128^3 GRF (contrast 10^6), b ~ N(0,1), rtol 1e-8."""
    _combo_pcg_parity(I.workload_grf(seed=0, n=128), 1e-8, 1e-7)


def test_layered128_combo_pcg_fp64():
    """The 128^3 layered workload (contrast 10^9, b = h^3).  Its true residual
    cannot go below eps |A||x| / |b| = 4e-7 in FP64, so the solve runs to 1e-6
    (both sides), and the two solutions must agree to 1e-5."""
    _combo_pcg_parity(I.workload_layered128(seed=0), 1e-6, 1e-5)
