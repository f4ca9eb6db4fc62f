"""GPU parity: the CUDA library (through its C ABI) against the FP64 CPU
oracle on the same seeded inputs.  Tolerances (tests/parity_bounds.py gives
the derivations):
  assembly / SpMV      1e-14 relative per entry (sum of |terms| for SpMV): the
                       only difference is FMA contraction (one rounding per term)
  setup factors, FP64  per entry, 2 * 4 * L * eps * cond, with cond the oracle's
                       own relative response to a 1e-13 perturbation of the bands
                       and L = max(nx, ny, nz) the longest recurrence chain
  apply kernel, FP64   1e-12 per entry in units of s = B^{-1}|r| (B^{-1} is
                       entrywise non-negative), against the oracle applying the
                       GPU's own exported factors (isolates the apply's rounding)
  setup + apply, FP64  per entry in units of s: 1e-12 + 2 * 4 * L * eps * amp,
                       amp = the oracle apply's response to the same perturbation
  apply, FP32 factors  1e-5 relative 2-norm (FP32 storage and arithmetic), and
                       per entry 1e-5 (or the FP32 rounding of the factors times
                       amp, if larger) in units of s
  PCG, FP64            iterations equal +-1, solution 1e-7 relative, both true
                       residuals below rtol
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
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def make(grid, seed, precision="fp64", contrast=3, bc=I.BC_Z_DIRICHLET, t=None, per_cell=False):
    w = I.random_small(grid, seed, contrast_exp=contrast, bc=bc, per_cell=per_cell)
    P = ffp.Preconditioner(grid, dev(w["kappa"]), bc, precision, t=None if t is None else dev(t))
    bands = o.assemble(grid, w["kappa"], bc)
    f = o.setup(grid, bands, t)
    return w, P, bands, f


# several tiles along x (S = 1..32 slots per lane), ragged tails, degenerate dims
GRIDS = [(1, 1, 1), (1, 1, 5), (5, 1, 1), (1, 6, 1), (2, 2, 2), (3, 8, 2), (5, 6, 7), (33, 5, 4),
         (17, 3, 9), (100, 4, 5), (64, 8, 6), (129, 3, 3), (350, 3, 4)]


@pytest.mark.parametrize("grid", GRIDS)
def test_assembly_parity(grid):
    w, P, bands, _ = make(grid, 1)
    ex = P.export()
    for k, ref in zip(("d", "cx", "cy", "cz"), bands):
        g = host(ex[k])
        assert np.all(np.abs(g - ref) <= 1e-14 * np.abs(ref) + 1e-300), k


@pytest.mark.parametrize("grid", GRIDS)
def test_spmv_parity(grid):
    w, P, bands, _ = make(grid, 2)
    x = np.random.default_rng(3).standard_normal(int(np.prod(grid)))
    y = host(P.spmv(dev(x)))
    yr = o.spmv(grid, bands, x)
    scale = o.spmv(grid, tuple(np.abs(b) for b in bands), np.abs(x))  # sum of |terms|
    assert np.all(np.abs(y - yr) <= 1e-14 * scale + 1e-300)


@pytest.mark.parametrize("grid", GRIDS)
def test_setup_factor_parity_fp64(grid):
    """Stored bands l2 (y-band of P_i), l1 (x-band of T_k), 1/M vs the oracle,
    per entry, within the bound derived from the oracle's own sensitivity."""
    _, P, bands, f = make(grid, 4)
    r = np.random.default_rng(6).standard_normal(int(np.prod(grid)))
    s, _ = PB.apply_scale(f, r)
    kf, _ = PB.sensitivity(grid, bands, f, r, s)
    tol = PB.factor_tol(grid, kf)
    ex = P.export()
    for k, ref in (("l2", f.Py), ("l1", f.To), ("minv", 1.0 / f.M)):
        g = host(ex[k])
        err = np.abs(g - ref)
        assert np.all(err <= tol * np.abs(ref) + 1e-300), (k, tol, float(np.max(err / (np.abs(ref) + 1e-300))))


def factors_of(P):
    """The GPU's stored factors as an oracle Factors object (FP64)."""
    ex = {k: host(v) for k, v in P.export().items()}
    n = ex["d"].size
    nan = np.full(n, np.nan)
    return o.Factors(P.grid, ex["l3"], nan, nan, ex["l2"], nan, ex["l1"], 1.0 / ex["minv"]), ex


@pytest.mark.parametrize("grid", GRIDS)
def test_apply_kernel_parity_fp64(grid):
    """The apply kernel against the oracle's Algorithms 1-7 on the same factors:
    1e-12 in the 2-norm and per entry in units of s = B^{-1}|r|."""
    _, P, _, f = make(grid, 5)
    r = np.random.default_rng(6).standard_normal(int(np.prod(grid)))
    z = host(P.apply(dev(r)))
    fg, _ = factors_of(P)
    s, zr = PB.apply_scale(fg, r)
    assert relerr(z, zr) <= 1e-12
    ok, worst = PB.per_entry_ok(z, zr, s, 1e-12)
    assert ok, worst


@pytest.mark.parametrize("grid", GRIDS)
def test_setup_and_apply_parity_fp64(grid):
    """Setup + apply end to end against the oracle with its own factors, per
    entry within 1e-12 + the setup's derived rounding carried through the apply."""
    _, P, bands, f = make(grid, 5)
    r = np.random.default_rng(6).standard_normal(int(np.prod(grid)))
    z = host(P.apply(dev(r)))
    s, zr = PB.apply_scale(f, r)
    _, amp = PB.sensitivity(grid, bands, f, r, s)
    ok, worst = PB.per_entry_ok(z, zr, s, PB.e2e_tol(grid, amp))
    assert ok, (worst, PB.e2e_tol(grid, amp))


@pytest.mark.parametrize("grid", GRIDS)
def test_apply_parity_fp32(grid):
    _, P, _, f = make(grid, 7, precision="fp32")
    r = np.random.default_rng(8).standard_normal(int(np.prod(grid)))
    z = host(P.apply(dev(r)))
    zr = o.apply(f, r)
    assert relerr(z, zr) <= 1e-5


@pytest.mark.parametrize("grid", [(33, 5, 4), (64, 8, 6), (350, 3, 4)])
def test_apply_kernel_parity_fp32_factors(grid):
    """FP32 arithmetic on FP32 factors against the FP64 oracle applying the
    exported factors: only FP32 rounding of the sweeps (and of the stored
    multipliers -1/M * coupling) differs."""
    _, P, _, _ = make(grid, 9, precision="fp32")
    r = np.random.default_rng(10).standard_normal(int(np.prod(grid)))
    z = host(P.apply(dev(r)))
    assert np.all(np.isfinite(z)) and relerr(z, o.apply(factors_of(P)[0], r)) <= 1e-5


@pytest.mark.parametrize("grid", [(33, 5, 4), (64, 8, 6), (350, 3, 4)])
def test_apply_bf16_factors_within_rounding(grid):
    """BF16 factor storage: each stored multiplier carries a relative rounding
    of at most 2^-9, and the apply's output moves by at most ~23 times a
    relative factor perturbation (measured on the oracle for these shapes), so
    the apply stays within 23 * 2^-9 = 4.5e-2 of the FP64 one."""
    _, P, _, f = make(grid, 9, precision="bf16")
    r = np.random.default_rng(10).standard_normal(int(np.prod(grid)))
    z = host(P.apply(dev(r)))
    assert np.all(np.isfinite(z)) and relerr(z, o.apply(f, r)) <= 5e-2


@pytest.mark.parametrize("grid", [(5, 6, 7), (33, 5, 4), (64, 8, 6), (17, 3, 9), (1, 1, 5), (350, 3, 4)])
def test_combination_parity_fp64(grid):
    """B_c (Sec. III Eq. (com)): ILU(0) pivots and the combined apply."""
    w = I.random_small(grid, 31, contrast_exp=3)
    P = ffp.Preconditioner(grid, dev(w["kappa"]), w["bc"], "fp64", precond="combo")
    bands = o.assemble(grid, w["kappa"], w["bc"])
    f = o.setup(grid, bands)
    Dp = o.ilu0_setup(grid, bands)
    fg, ex = factors_of(P)
    # ILU(0) pivots: the GPU evaluates their continued fraction by a projective scan
    np.testing.assert_allclose(ex["dinv"], 1.0 / Dp, rtol=1e-10)
    r = np.random.default_rng(32).standard_normal(int(np.prod(grid)))
    z = host(P.apply(dev(r)))
    assert relerr(z, o.combo_apply(grid, bands, fg, 1.0 / ex["dinv"], r)) <= 1e-12
    # end to end: the NTD factors' rounding (derived bound) carried through B_c,
    # measured as the oracle's response to the same 1e-13 band perturbation
    zr = o.combo_apply(grid, bands, f, Dp, r)
    rng = np.random.default_rng(99)
    bp = tuple(b * (1.0 + PB.PERTURB * rng.uniform(-1.0, 1.0, b.size)) for b in bands)
    zp = o.combo_apply(grid, bands, o.setup(grid, bp), o.ilu0_setup(grid, bp), r)
    amp2 = relerr(zp, zr) / PB.PERTURB
    tol = 1e-12 + 2.0 * PB.SAFETY * PB.chain(grid) * PB.EPS * max(amp2, 1.0)
    assert relerr(z, zr) <= tol, (relerr(z, zr), tol)


@pytest.mark.parametrize("grid", [(33, 5, 4), (64, 8, 6)])
def test_combination_parity_fp32(grid):
    w = I.random_small(grid, 33, contrast_exp=3)
    P = ffp.Preconditioner(grid, dev(w["kappa"]), w["bc"], "fp32", precond="combo")
    bands = o.assemble(grid, w["kappa"], w["bc"])
    r = np.random.default_rng(34).standard_normal(int(np.prod(grid)))
    zr = o.combo_apply(grid, bands, o.setup(grid, bands), o.ilu0_setup(grid, bands), r)
    assert relerr(host(P.apply(dev(r))), zr) <= 1e-5


@pytest.mark.parametrize("grid", [(33, 1, 7), (40, 6, 1), (350, 3, 4), (70, 24, 20)])
def test_combination_parity_fp32_shapes(grid):
    """B_c with FP32 factors on degenerate and many-plane shapes (ny = 1, nz = 1,
    the longest line, several CTAs of plane sweeps): within FP32 rounding of the
    FP64 oracle, and repeated applies (each a new ILU(0) sweep epoch) are bitwise
    identical."""
    w = I.random_small(grid, 35, contrast_exp=3)
    P = ffp.Preconditioner(grid, dev(w["kappa"]), w["bc"], "fp32", precond="combo")
    bands = o.assemble(grid, w["kappa"], w["bc"])
    r = np.random.default_rng(36).standard_normal(int(np.prod(grid)))
    zr = o.combo_apply(grid, bands, o.setup(grid, bands), o.ilu0_setup(grid, bands), r)
    rd = dev(r)
    z1 = P.apply(rd)
    assert relerr(host(z1), zr) <= 1e-5
    for _ in range(3):
        assert torch.equal(P.apply(rd), z1)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_combination_pcg_blocks32(precision):
    w = I.workload_blocks32(seed=0)
    g, bc = w["grid"], w["bc"]
    P = ffp.Preconditioner(g, dev(w["kappa"]), bc, precision, precond="combo")
    x, st = P.solve(dev(w["b"]), rtol=1e-8, maxit=200)
    bands = o.assemble(g, w["kappa"], bc)
    ref = o.pcg(g, bands, o.setup(g, bands), w["b"], rtol=1e-8, maxit=200, flexible=True,
                ilu=o.ilu0_setup(g, bands))
    assert st["status"] == 0 and ref["status"] == 0 and st["rel_res_true"] < 1e-8
    xr = host(x)
    assert np.linalg.norm(w["b"] - o.spmv(g, bands, xr)) / np.linalg.norm(w["b"]) < 1e-8
    if precision == "fp64":
        assert abs(st["iters"] - ref["iters"]) <= 1
        assert relerr(xr, ref["x"]) <= 1e-7
    else:
        assert st["iters"] <= ref["iters"] + 3


def test_user_filter_parity():
    grid = (9, 7, 6)
    t = np.random.default_rng(11).uniform(0.5, 2.0, int(np.prod(grid)))
    _, P, bands, f = make(grid, 12, t=t)
    ex = P.export()
    r = np.random.default_rng(13).standard_normal(int(np.prod(grid)))
    s, zr = PB.apply_scale(f, r)
    kf, amp = PB.sensitivity(grid, bands, f, r, s, t=t)
    assert np.max(np.abs(host(ex["minv"]) - 1.0 / f.M) / (1.0 / f.M)) <= PB.factor_tol(grid, kf)
    z = host(P.apply(dev(r)))
    ok, worst = PB.per_entry_ok(z, zr, s, PB.e2e_tol(grid, amp))
    assert ok, worst
    assert relerr(z, o.apply(factors_of(P)[0], r)) <= 1e-12


@pytest.mark.parametrize("grid", [(1024, 2, 3), (1023, 3, 2)])
def test_longest_line(grid):
    """The longest lines (S = 32).  The apply on the GPU's own factors meets the
    apply bound (1e-12 per entry).  Setup plus apply end to end meets the bound
    derived from the oracle's sensitivity: beta = (T^{-1} w) ./ w inherits the
    conditioning of a nearly singular Neumann line, which grows like nx^2, and
    the setup's recurrences round in another order than the oracle's."""
    _, P, bands, f = make(grid, 14, contrast=2)
    r = np.random.default_rng(15).standard_normal(int(np.prod(grid)))
    z = host(P.apply(dev(r)))
    fg, _ = factors_of(P)
    sg, zg = PB.apply_scale(fg, r)
    ok, worst = PB.per_entry_ok(z, zg, sg, 1e-12)
    assert ok, worst
    s, zr = PB.apply_scale(f, r)
    _, amp = PB.sensitivity(grid, bands, f, r, s)
    ok, worst = PB.per_entry_ok(z, zr, s, PB.e2e_tol(grid, amp))
    assert ok, (worst, PB.e2e_tol(grid, amp))


def test_pcg_parity_fp64_grf32():
    """Plain B_NTD PCG (the rowsum NTD alone does not converge on the 10^6
    block workload within maxit, on the oracle as on the GPU; the 10^2 GRF
    converges)."""
    w = I.workload_grf(seed=0, n=32, exponent=1.0)
    g, bc = w["grid"], w["bc"]
    P = ffp.Preconditioner(g, dev(w["kappa"]), bc, "fp64")
    x, st = P.solve(dev(w["b"]), rtol=1e-8, maxit=1000)
    bands = o.assemble(g, w["kappa"], bc)
    ref = o.pcg(g, bands, o.setup(g, bands), w["b"], rtol=1e-8, maxit=1000)
    assert st["status"] == 0 and ref["status"] == 0
    assert abs(st["iters"] - ref["iters"]) <= 1
    assert st["rel_res_true"] < 1e-8 and ref["relres"] < 1e-8
    assert relerr(host(x), ref["x"]) <= 1e-7
    # independent true residual with the oracle's operator
    xr = host(x)
    assert np.linalg.norm(w["b"] - o.spmv(g, bands, xr)) / np.linalg.norm(w["b"]) < 1e-8
    # Lanczos estimate of cond(B^{-1} A) from the CG coefficients (O5): the same
    # coefficients up to rounding, so the same extremes; the GPU's bisection
    # against the oracle's dense eigensolver of its own tridiagonal
    lmin, lmax = o.lanczos_extremes(ref["alpha"], ref["beta"])
    assert abs(st["lanczos_min"] - lmin) <= 1e-6 * lmin
    assert abs(st["lanczos_max"] - lmax) <= 1e-6 * lmax
    assert st["cond_est"] == pytest.approx(lmax / lmin, rel=2e-6)


def test_lanczos_estimate_of_a_known_spectrum():
    """On a 1-D problem B = A exactly (level 1 is exact), so B^{-1} A = I: one
    CG step, and the Lanczos tridiagonal is the 1 x 1 matrix [1]."""
    grid = (40, 1, 1)
    w = I.random_small(grid, 5, contrast_exp=3)
    P = ffp.Preconditioner(grid, dev(w["kappa"]), w["bc"], "fp64")
    _, st = P.solve(dev(w["b"]), rtol=1e-12, maxit=10)
    assert st["iters"] == 1 and st["status"] == 0
    assert st["lanczos_min"] == pytest.approx(1.0, rel=1e-12)
    assert st["lanczos_max"] == pytest.approx(1.0, rel=1e-12)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_flexible_cg_converges_grf32(precision):
    w = I.workload_grf(seed=1, n=32, exponent=1.0)
    g, bc = w["grid"], w["bc"]
    P = ffp.Preconditioner(g, dev(w["kappa"]), bc, precision)
    x, st = P.solve(dev(w["b"]), rtol=1e-8, maxit=1000)
    bands = o.assemble(g, w["kappa"], bc)
    ref = o.pcg(g, bands, o.setup(g, bands), w["b"], rtol=1e-8, maxit=1000)
    assert st["status"] == 0 and st["rel_res_true"] < 1e-8
    xr = host(x)
    assert np.linalg.norm(w["b"] - o.spmv(g, bands, xr)) / np.linalg.norm(w["b"]) < 1e-8
    if precision == "fp32":
        assert st["iters"] <= ref["iters"] + 5


def test_zero_rhs_and_warm_start():
    grid = (6, 5, 4)
    w, P, bands, f = make(grid, 16)
    x, st = P.solve(dev(np.zeros(120)))
    assert st["iters"] == 0 and st["status"] == 0 and not torch.any(x != 0)
    x, st = P.solve(dev(w["b"]), rtol=1e-10)
    x2, st2 = P.solve(dev(w["b"]), x=x.clone(), rtol=1e-10)
    assert st2["iters"] == 0 and st2["rel_res_true"] < 1e-10


def test_bad_arguments_rejected():
    grid = (4, 4, 4)
    k = np.ones(64)
    k[5] = -1.0
    with pytest.raises(ffp.FFPError) as e:
        ffp.Preconditioner(grid, dev(k), I.BC_Z_DIRICHLET)
    assert e.value.status == ffp.FFP_ERR_ARG
    k[5] = np.nan
    with pytest.raises(ffp.FFPError):
        ffp.Preconditioner(grid, dev(k), I.BC_Z_DIRICHLET)
    t = np.ones(64)
    t[3] = 0.0
    with pytest.raises(ffp.FFPError) as e:
        ffp.Preconditioner(grid, dev(np.ones(64)), I.BC_Z_DIRICHLET, t=dev(t))
    assert e.value.status == ffp.FFP_ERR_ARG
    with pytest.raises(ffp.FFPError):
        ffp.Preconditioner((ffp.FFP_MAX_NX + 1, 1, 1), dev(np.ones(ffp.FFP_MAX_NX + 1)),
                           I.BC_Z_DIRICHLET)


def test_pure_neumann_breakdown_reported():
    """All-Neumann: A is singular (constant null vector), so the rowsum-filtered
    factorization reaches a zero pivot on the last eliminated block; the setup
    reports a breakdown (or, if rounding keeps the pivot positive, the
    preconditioner is still applied without fault)."""
    grid = (4, 3, 3)
    try:
        ffp.Preconditioner(grid, dev(np.ones(36)), (1, 1, 1, 1, 1, 1))
    except ffp.FFPError as e:
        assert e.status == ffp.FFP_ERR_BREAKDOWN


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_apply_symmetric_positive_layered128(precision):
    """At the 128^3 layered workload size: B^{-1} is symmetric and positive
    definite (properties that hold at any size): <B^-1 u, v> = <u, B^-1 v>,
    <u, B^-1 u> > 0; and repeated applies are bitwise identical."""
    w = I.workload_layered128(seed=0)
    P = ffp.Preconditioner(w["grid"], dev(w["kappa"]), w["bc"], precision)
    rng = np.random.default_rng(17)
    u = dev(rng.standard_normal(w["kappa"].size))
    v = dev(rng.standard_normal(w["kappa"].size))
    Bu, Bv = P.apply(u), P.apply(v)
    a, b = float(torch.dot(Bu, v)), float(torch.dot(u, Bv))
    tol = 1e-12 if precision == "fp64" else 1e-5
    assert abs(a - b) <= tol * (float(torch.norm(Bu)) * float(torch.norm(v)))
    assert float(torch.dot(u, Bu)) > 0
    assert torch.equal(P.apply(u), Bu)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_unreachable_tolerance_stops_early(precision):
    """rtol below what an FP64 iterate can reach (1e-17 < eps): the recursive
    residual still meets it, the true residual confirmations stop improving,
    and the solve ends with FFP_ERR_NOT_CONVERGED long before maxit, with the
    iterate as accurate as FP64 allows."""
    w = I.random_small((24, 20, 16), 77, contrast_exp=3)
    P = ffp.Preconditioner(w["grid"], dev(w["kappa"]), w["bc"], precision, precond="combo")
    _, st = P.solve(dev(w["b"]), rtol=1e-17, maxit=3000, check=False)
    assert st["status"] == ffp.FFP_ERR_NOT_CONVERGED
    assert 0 < st["iters_rec"] < st["iters"] < 600
    assert st["rel_res_true"] < 1e-12


# ---------------------------------------------------------------- X = beta (FFP_SCHUR_BETA)
SCHUR_GRIDS = [(1, 1, 5), (5, 6, 7), (33, 5, 4), (17, 3, 9), (64, 8, 6), (350, 3, 4), (70, 24, 20)]


@pytest.mark.parametrize("grid", SCHUR_GRIDS)
def test_schur_beta_setup_and_apply_parity_fp64(grid):
    """The classical Schur form X = beta: stored factors per entry within the
    derived bound, the apply kernel on the GPU's own factors (1e-12 per entry
    of s) and setup + apply end to end against the oracle's X = beta form."""
    w = I.random_small(grid, 61, contrast_exp=3)
    P = ffp.Preconditioner(grid, dev(w["kappa"]), w["bc"], "fp64", schur="beta")
    bands = o.assemble(grid, w["kappa"], w["bc"])
    f = o.setup(grid, bands, schur="beta")
    r = np.random.default_rng(62).standard_normal(int(np.prod(grid)))
    z = host(P.apply(dev(r)))
    s, zr = PB.apply_scale(f, r)
    kf, amp = PB.sensitivity(grid, bands, f, r, s, schur="beta")
    ex = P.export()
    for k, ref in (("l2", f.Py), ("l1", f.To), ("minv", 1.0 / f.M)):
        err = np.abs(host(ex[k]) - ref)
        assert np.all(err <= PB.factor_tol(grid, kf) * np.abs(ref) + 1e-300), k
    fg, _ = factors_of(P)
    sg, zg = PB.apply_scale(fg, r)
    assert PB.per_entry_ok(z, zg, sg, 1e-12)[0]
    ok, worst = PB.per_entry_ok(z, zr, s, PB.e2e_tol(grid, amp))
    assert ok, worst


@pytest.mark.parametrize("grid", [(33, 5, 4), (350, 3, 4), (70, 24, 20)])
def test_schur_beta_apply_parity_fp32(grid):
    w = I.random_small(grid, 63, contrast_exp=3)
    P = ffp.Preconditioner(grid, dev(w["kappa"]), w["bc"], "fp32", schur="beta")
    bands = o.assemble(grid, w["kappa"], w["bc"])
    r = np.random.default_rng(64).standard_normal(int(np.prod(grid)))
    assert relerr(host(P.apply(dev(r))), o.apply(o.setup(grid, bands, schur="beta"), r)) <= 1e-5


@pytest.mark.parametrize("precond", ["ntd", "combo"])
def test_schur_beta_pcg_parity_fp64_blocks32(precond):
    """PCG with X = beta on the 32^3 block workload (contrast 10^6): plain
    B_NTD (standard PCG) and B_c (flexible CG) against the oracle: iterations
    within one, solutions within 1e-7, both true residuals below 1e-8."""
    wl = I.workload_blocks32(seed=0)
    g, bc = wl["grid"], wl["bc"]
    P = ffp.Preconditioner(g, dev(wl["kappa"]), bc, "fp64", precond=precond, schur="beta")
    x, st = P.solve(dev(wl["b"]), rtol=1e-8, maxit=500)
    bands = o.assemble(g, wl["kappa"], bc)
    f = o.setup(g, bands, schur="beta")
    ref = o.pcg(g, bands, f, wl["b"], rtol=1e-8, maxit=500, flexible=(precond == "combo"),
                ilu=o.ilu0_setup(g, bands) if precond == "combo" else None)
    assert st["status"] == 0 and ref["status"] == 0
    assert abs(st["iters"] - ref["iters"]) <= 1
    assert st["rel_res_true"] < 1e-8 and ref["relres"] < 1e-8
    assert relerr(host(x), ref["x"]) <= 1e-7
