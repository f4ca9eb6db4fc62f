"""Batched solves (include/ffp.h ffp_batch_*) against standalone solves and the
oracle.

A batched pair runs the same kernels, line slot count, reduction partition and
control flow as its standalone ffp_pcg_solve, so its iteration count must be
equal and its solution equal to 1e-12 relative (the only allowed difference is
none at all in practice; the bound leaves room for nothing but rounding).  The
launch configuration (ILU(0) warps per CTA, parallel or sequential groups) must
not change any result.  One pair is also checked against the FP64 oracle's PCG
with the PCG tolerances of the single-instance tests (iterations +-1, solution
1e-7), and the full 64-instance workload is checked by independent true
residuals on sampled pairs and by standalone solves of sampled pairs.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as o
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


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def relerr(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


# slot counts (apply S, ILU S): (1,1) (2,2) (3,3) (1,1) (1,2); one single-plane instance
GRIDS = [(8, 6, 5), (40, 9, 7), (70, 5, 12), (17, 11, 1), (33, 4, 9)]
NRHS = 2


def instances(contrast):
    out = []
    for i, g in enumerate(GRIDS):
        w = I.random_small(g, 100 + i, contrast_exp=contrast)
        rng = np.random.default_rng(200 + i)
        bs = [rng.standard_normal(int(np.prod(g))) for _ in range(NRHS)]
        out.append((w, bs))
    return out


def make_batch(inst, precision, precond):
    return ffp.Batch([w["grid"] for w, _ in inst], [dev(w["kappa"]) for w, _ in inst],
                     [w["bc"] for w, _ in inst], nrhs=NRHS, precision=precision, precond=precond)


def rhs_list(inst):
    return [dev(b) for _, bs in inst for b in bs]


CASES = [("fp64", "combo", 3), ("fp32", "combo", 3), ("bf16", "combo", 3), ("fp64", "ntd", 1),
         ("fp32", "ntd", 1)]


@pytest.mark.parametrize("rhs_per_cta", [1, 2])
@pytest.mark.parametrize("precision,precond,contrast", CASES)
def test_pairs_equal_standalone_solves(precision, precond, contrast, rhs_per_cta):
    """rhs_per_cta = 2: the two right-hand sides of an instance share one chain of
    apply CTAs (one factor stage ring, two pairs of compute warps)."""
    inst = instances(contrast)
    bat = make_batch(inst, precision, precond)
    assert bat.info()["groups"] == 4
    bat.set_config(4, 1, rhs_per_cta)
    xs, stats = bat.solve(rhs_list(inst), rtol=1e-8, maxit=300, check=False)
    for i, (w, bs) in enumerate(inst):
        P = ffp.Preconditioner(w["grid"], dev(w["kappa"]), w["bc"], precision, precond=precond)
        for j, b in enumerate(bs):
            x, st = P.solve(dev(b), rtol=1e-8, maxit=300, check=False)
            s = stats[i * NRHS + j]
            assert s["status"] == st["status"] and s["iters"] == st["iters"], (i, j, s, st)
            assert relerr(host(xs[i * NRHS + j]), host(x)) <= 1e-12, (i, j)
            if st["status"] == 0:
                assert s["rel_res_true"] < 1e-8


def test_configuration_changes_no_result():
    """ILU(0) warps, parallel or sequential groups and one or two right-hand
    sides per apply CTA give bitwise identical solves."""
    inst = instances(3)
    bat = make_batch(inst, "fp32", "combo")
    out = []
    for warps, branches, nr in [(2, 0, 1), (8, 1, 2), (4, 1, 1), (2, 1, 2), (4, 0, 2)]:
        bat.set_config(warps, branches, nr)
        xs, stats = bat.solve(rhs_list(inst), rtol=1e-8, maxit=300)
        out.append(([host(x) for x in xs], [s["iters"] for s in stats]))
    for xs, its in out[1:]:
        assert its == out[0][1]
        for a, b in zip(xs, out[0][0]):
            assert np.array_equal(a, b)


def test_tune_and_cache(tmp_path):
    inst = instances(3)
    cache = str(tmp_path / "tune.txt")
    bat = make_batch(inst, "fp32", "combo")
    c1 = bat.tune(cache)
    assert c1["from_cache"] == 0 and c1["ms"] > 0 and 1 <= c1["ilu_warps"] <= 8
    assert open(cache).read().count("\n") == 1
    bat2 = make_batch(inst, "fp32", "combo")
    c2 = bat2.tune(cache)
    assert c2["from_cache"] == 1
    assert (c2["ilu_warps"], c2["branches"], c2["rhs_per_cta"]) == (c1["ilu_warps"], c1["branches"],
                                                                     c1["rhs_per_cta"])
    assert c1["rhs_per_cta"] in (1, 2)
    # the tuned batch still solves exactly as an untuned one
    xs, st = bat.solve(rhs_list(inst), rtol=1e-8, maxit=300)
    ref = make_batch(inst, "fp32", "combo")
    xr, sr = ref.solve(rhs_list(inst), rtol=1e-8, maxit=300)
    assert [s["iters"] for s in st] == [s["iters"] for s in sr]
    assert all(np.array_equal(host(a), host(b)) for a, b in zip(xs, xr))


def test_pair_against_oracle():
    inst = instances(3)
    bat = make_batch(inst, "fp64", "combo")
    xs, stats = bat.solve(rhs_list(inst), rtol=1e-8, maxit=300)
    for i in (1, 2):
        w, bs = inst[i]
        g = w["grid"]
        bands = o.assemble(g, w["kappa"], w["bc"])
        ref = o.pcg(g, bands, o.setup(g, bands), bs[1], rtol=1e-8, maxit=300, flexible=True,
                    ilu=o.ilu0_setup(g, bands))
        s = stats[i * NRHS + 1]
        assert ref["status"] == 0 and s["status"] == 0
        assert abs(s["iters"] - ref["iters"]) <= 1
        assert relerr(host(xs[i * NRHS + 1]), ref["x"]) <= 1e-7
        xr = host(xs[i * NRHS + 1])
        assert np.linalg.norm(bs[1] - o.spmv(g, bands, xr)) / np.linalg.norm(bs[1]) < 1e-8


def test_zero_rhs_warm_start_and_maxit():
    inst = instances(3)
    bat = make_batch(inst, "fp32", "combo")
    bs = rhs_list(inst)
    bs[3] = torch.zeros_like(bs[3])
    xs, stats = bat.solve(bs, rtol=1e-8, maxit=300)
    assert stats[3]["iters"] == 0 and stats[3]["status"] == 0 and not torch.any(xs[3] != 0)
    assert all(s["iters"] > 0 for k, s in enumerate(stats) if k != 3)
    # warm start from the solutions: nothing left to do
    xs2, stats2 = bat.solve(bs, xs=[x.clone() for x in xs], rtol=1e-8, maxit=300)
    assert all(s["iters"] == 0 for s in stats2)
    # maxit stops every pair at the same iterate as a standalone solve
    xs3, stats3 = bat.solve(bs, rtol=1e-8, maxit=2, check=False)
    w, b = inst[2][0], inst[2][1][0]
    P = ffp.Preconditioner(w["grid"], dev(w["kappa"]), w["bc"], "fp32", precond="combo")
    x, st = P.solve(dev(b), rtol=1e-8, maxit=2, check=False)
    assert st["status"] == ffp.FFP_ERR_NOT_CONVERGED
    assert stats3[4]["status"] == ffp.FFP_ERR_NOT_CONVERGED and stats3[4]["iters"] == 2
    assert relerr(host(xs3[4]), host(x)) <= 1e-12


def test_bad_arguments_rejected():
    assert ffp.batch_workspace_bytes([(1025, 2, 2)], 1) == 0
    assert ffp.batch_workspace_bytes([(4, 4, 4)], 0) == 0
    assert ffp.batch_workspace_bytes([(4, 4, 4)], 65536) == 0
    k = dev(np.ones(64))
    with pytest.raises(ffp.FFPError):
        ffp.Batch([(4, 4, 4)], [k], [(1, 1, 1, 1, 0, 7)])
    bat = ffp.Batch([(4, 4, 4)], [k], [(1, 1, 1, 1, 0, 0)], nrhs=1)
    with pytest.raises(ValueError):
        bat.solve([dev(np.ones(64))] * 2)
    with pytest.raises(ffp.FFPError):
        bat.set_config(0, 1)
    # one instance with a bad kappa (negative, NaN) or filter (t <= 0) fails the whole batch
    for bad in (-1.0, np.nan):
        kb = np.ones(60)
        kb[7] = bad
        with pytest.raises(ffp.FFPError) as e:
            ffp.Batch([(4, 4, 4), (5, 4, 3)], [k, dev(kb)], [I.BC_Z_DIRICHLET] * 2)
        assert e.value.status == ffp.FFP_ERR_ARG
    tb = np.ones(60)
    tb[3] = 0.0
    with pytest.raises(ffp.FFPError) as e:
        ffp.Batch([(4, 4, 4), (5, 4, 3)], [k, dev(np.ones(60))], [I.BC_Z_DIRICHLET] * 2,
                  ts=[None, dev(tb)])
    assert e.value.status == ffp.FFP_ERR_ARG


def test_full_batched_workload_sampled():
    """The 64 x [48,160]^3 workload with 4 right-hand sides each, FP32 factors
    and B_c, in the launch configuration the benchmark times: every pair
    converges with an independent true residual below rtol on sampled pairs,
    and sampled pairs equal their standalone solves."""
    ws = I.workload_batched(seed=0)
    bat = ffp.Batch([w["grid"] for w in ws], [dev(w["kappa"]) for w in ws], [w["bc"] for w in ws],
                    nrhs=4, precision="fp32", precond="combo")
    bat.tune()
    bs = [dev(b) for w in ws for b in w["b"]]
    xs, stats = bat.solve(bs, rtol=1e-8, maxit=400)
    assert all(s["status"] == 0 and s["rel_res_true"] < 1e-8 for s in stats)
    for p in (0, 77, 255):
        w = ws[p // 4]
        g = w["grid"]
        bands = o.assemble(g, w["kappa"], w["bc"])
        b = w["b"][p % 4]
        assert np.linalg.norm(b - o.spmv(g, bands, host(xs[p]))) / np.linalg.norm(b) < 1e-8
        P = ffp.Preconditioner(g, dev(w["kappa"]), w["bc"], "fp32", precond="combo")
        x, st = P.solve(dev(b), rtol=1e-8, maxit=400)
        assert st["iters"] == stats[p]["iters"]
        assert relerr(host(xs[p]), host(x)) <= 1e-12


def test_unreachable_tolerance_pairs_equal_standalone():
    """The stagnation stop (three confirmations that do not halve the true
    residual) decides per pair exactly as the single-instance driver does."""
    inst = instances(3)
    bat = make_batch(inst, "fp32", "combo")
    _, stats = bat.solve(rhs_list(inst), rtol=1e-17, maxit=3000, check=False)
    for i, (w, bs) in enumerate(inst):
        P = ffp.Preconditioner(w["grid"], dev(w["kappa"]), w["bc"], "fp32", precond="combo")
        for j, b in enumerate(bs):
            _, st = P.solve(dev(b), rtol=1e-17, maxit=3000, check=False)
            s = stats[i * NRHS + j]
            # tiny grids may meet even 1e-17 exactly; the others must stop on the stall rule
            assert s["status"] == st["status"] and st["status"] in (0, ffp.FFP_ERR_NOT_CONVERGED), (i, j, s, st)
            assert s["iters"] == st["iters"] < 600 and s["iters_rec"] == st["iters_rec"], (i, j)
