"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix
(no GPU).  Each test names the passage it pins and the property used.

The paper prints no worked numerical example, so the pins are: hand-derived
fixtures (tests/golden), closed forms and special cases that reduce to a
textbook routine (1-D: B = A, a banded solve), dense brute force on small
grids, identities that follow from the definitions (symmetry, level-2
filtering, the closed-form level-3 filtering defect), and PCG theory
(monotone A-norm error, Lanczos extremes).
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import oracle as o
from paper_1909_09771_gb300 import inputs as I
from tests import dense_ref as D

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_fixture(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


def _case(grid, seed, contrast=3, bc=I.BC_Z_DIRICHLET, per_cell=False, t=None):
    w = I.random_small(grid, seed, contrast_exp=contrast, bc=bc, per_cell=per_cell)
    bands = o.assemble(grid, w["kappa"], bc)
    f = o.setup(grid, bands, t)
    return w, bands, f


def _binv(f, n):
    return np.column_stack([o.apply(f, e) for e in np.eye(n)])


# ----------------------------------------------------------------- assembly (P8)

def test_golden_two_cell_assembly():
    """Sec. I Eq. (2), FV reading: hand-derived 2-cell operator."""
    g, bc, kap, d_exp, cx_exp = _read_fixture("two_cell_assembly.txt")
    grid = tuple(int(v) for v in g)
    d, cx, cy, cz = o.assemble(grid, np.array(kap), [int(v) for v in bc])
    np.testing.assert_allclose(d, d_exp, rtol=1e-15)
    np.testing.assert_allclose(cx, cx_exp, rtol=1e-15)
    assert np.all(cy == 0) and np.all(cz == 0)


def test_assembly_poisson_equals_kron_laplacian():
    """kappa = 1: the FV operator is h * (kron-sum of 1-D second differences)
    with a doubled end coefficient on Dirichlet faces."""
    nx, ny, nz = 4, 3, 5
    bc = (1, 0, 0, 1, 0, 0)
    d, cx, cy, cz = o.assemble((nx, ny, nz), np.ones(nx * ny * nz), bc)
    A = D.dense_A((nx, ny, nz), (d, cx, cy, cz))

    def lap1(n, h, lo_dir, hi_dir, area):
        T = np.zeros((n, n))
        for i in range(n - 1):
            T[i, i] += 1; T[i + 1, i + 1] += 1; T[i, i + 1] -= 1; T[i + 1, i] -= 1
        if lo_dir: T[0, 0] += 2
        if hi_dir: T[-1, -1] += 2
        return T * area / h

    hx, hy, hz = 1 / nx, 1 / ny, 1 / nz
    Lx = lap1(nx, hx, bc[0] == 0, bc[1] == 0, hy * hz)
    Ly = lap1(ny, hy, bc[2] == 0, bc[3] == 0, hx * hz)
    Lz = lap1(nz, hz, bc[4] == 0, bc[5] == 0, hx * hy)
    K = (np.kron(np.eye(nz), np.kron(np.eye(ny), Lx)) + np.kron(np.eye(nz), np.kron(Ly, np.eye(nx)))
         + np.kron(Lz, np.eye(nx * ny)))
    np.testing.assert_allclose(A, K, rtol=1e-13, atol=1e-13)


def test_assembly_symmetric_rowsum_zero_under_neumann():
    """A symmetric positive definite; rows whose cell has no Dirichlet face sum to 0."""
    grid = (5, 4, 6)
    w = I.random_small(grid, 3, contrast_exp=3)
    bands = o.assemble(grid, w["kappa"], I.BC_Z_DIRICHLET)
    A = D.dense_A(grid, bands)
    np.linalg.cholesky(A)
    rs = A.sum(axis=1).reshape(grid[2], grid[1], grid[0])
    inner = rs[1:-1]
    assert np.max(np.abs(inner)) <= 1e-12 * np.max(np.abs(A))
    assert np.all(rs[0] > 0) and np.all(rs[-1] > 0)


def test_assembly_rejects_bad_kappa():
    with pytest.raises(o.OracleError):
        o.assemble((2, 2, 2), np.array([1, 1, 1, 0, 1, 1, 1, 1.0]), I.BC_Z_DIRICHLET)


# ----------------------------------------------------------------- level 1 (P1, P2)

def test_golden_three_cell_twisted_pivots():
    """Sec. II-A level-1 recurrence for M_i with the twist at m = 1."""
    g, bc, kap, M_exp, rhs, x_exp = _read_fixture("three_cell_twisted.txt")
    grid = tuple(int(v) for v in g[:3])
    bands = o.assemble(grid, np.array(kap), [int(v) for v in bc], lengths=g[3:])
    f = o.setup(grid, bands)
    np.testing.assert_allclose(f.M, M_exp, rtol=1e-15)
    np.testing.assert_allclose(o.apply(f, np.array(rhs)), x_exp, rtol=1e-14)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 16, 33])
def test_1d_B_equals_A_banded_solve(n):
    """ny = nz = 1: levels 2 and 3 are trivial and the level-1 factorization is
    exact, so B = A and the apply equals a banded LAPACK solve (P1)."""
    rng = np.random.default_rng(n)
    kappa = np.power(10.0, rng.uniform(-3, 3, n))
    bands = o.assemble((n, 1, 1), kappa, (0, 1, 1, 1, 1, 1))
    f = o.setup((n, 1, 1), bands)
    d, cx = bands[0], bands[1]
    ab = np.zeros((3, n))
    ab[0, 1:] = cx[:-1]
    ab[1] = d
    ab[2, :-1] = cx[:-1]
    r = rng.standard_normal(n)
    x = o.apply(f, r)
    xl = sla.solve_banded((1, 1), ab, r)
    A = D.dense_A((n, 1, 1), bands)
    # both solves are backward stable: tiny backward error, forward error within cond(A) * eps
    assert np.linalg.norm(A @ x - r) <= 1e-14 * np.linalg.norm(A, 2) * np.linalg.norm(x)
    bound = 8 * n * np.linalg.cond(A) * np.finfo(float).eps
    assert np.linalg.norm(x - xl) <= max(bound, 1e-14) * np.linalg.norm(xl)
    # PCG with B = A converges in one iteration (mild contrast so that the
    # residual of the exact solve is itself below rtol)
    kap2 = np.power(10.0, rng.uniform(-1, 1, n))
    bands2 = o.assemble((n, 1, 1), kap2, (0, 1, 1, 1, 1, 1))
    res = o.pcg((n, 1, 1), bands2, o.setup((n, 1, 1), bands2), r, rtol=1e-10)
    assert res["status"] == 0 and res["iters"] == 1 and res["relres"] < 1e-12


def test_pivots_reproduce_line_tridiagonals():
    """(M + L1) M^{-1} (M + U1) equals every stored T_k (P2): the twisted
    pivots are consistent with the T bands."""
    grid = (7, 5, 4)
    _, _, f = _case(grid, 11)
    nx = grid[0]
    for k in range(grid[1] * grid[2]):
        s = slice(k * nx, (k + 1) * nx)
        T = D.tridiag(f.Td[s], f.To[s])
        np.testing.assert_allclose(D.line_T_from_pivots(f.M[s], f.To[s]), T, rtol=1e-13,
                                   atol=1e-13 * np.abs(T).max())
        # and T_k^{-1} via the oracle's level-1 solve equals a dense solve
    assert np.all(f.M > 0)


# ----------------------------------------------------------------- the factorization (P4, P5, P7)

GRIDS = [(5, 6, 7), (3, 8, 2), (4, 4, 4), (1, 1, 1), (2, 2, 2), (3, 3, 3), (2, 3, 1), (1, 4, 5),
         (6, 1, 3)]


@pytest.mark.parametrize("grid", GRIDS)
def test_sweep_equals_dense_factorization(grid):
    """Algorithms 1-7 applied to unit vectors give the columns of B^{-1},
    where B = (B_P + L3) B_P^{-1} (B_P + U3), B_P = (T + L2) T^{-1} (T + U2),
    T = (M + L1) M^{-1} (M + U1), built densely from the stored bands (P4)."""
    n = int(np.prod(grid))
    _, _, f = _case(grid, 5)
    B, _ = D.dense_B(grid, f)
    Bi = _binv(f, n)
    err = np.linalg.norm(Bi @ B - np.eye(n)) / np.sqrt(n)
    assert err < 1e-11


@pytest.mark.parametrize("grid,contrast", [((5, 6, 7), 3), ((4, 5, 3), 6), ((6, 6, 6), 6)])
def test_B_symmetric_positive_definite(grid, contrast):
    """B symmetric, positive definite (Cholesky), eigenvalues of B^{-1}A in
    (0, ~1] (P5), with per-cell kappa contrast up to 10^12."""
    n = int(np.prod(grid))
    w, bands, f = _case(grid, 7, contrast=contrast // 2, per_cell=True)
    Bi = _binv(f, n)
    assert np.linalg.norm(Bi - Bi.T) <= 1e-12 * np.linalg.norm(Bi)
    np.linalg.cholesky(0.5 * (Bi + Bi.T))
    A = D.dense_A(grid, bands)
    ev = sla.eigh(A, np.linalg.inv(0.5 * (Bi + Bi.T)), eigvals_only=True)
    assert ev.min() > 0 and ev.max() < 1.1


@pytest.mark.parametrize("grid", [(3, 3, 3), (4, 3, 5), (2, 5, 4)])
def test_exact_twisted_block_lu_reproduces_A(grid):
    """With exact dense inverses in the plane recurrence (Sec. II-A, the
    unapproximated P_i), (P + L3)(I + P^{-1} U3) = A: pins the twisted block
    structure the dense B of the other pins relies on (P7)."""
    nx, ny, nz = grid
    nxy = nx * ny
    w = I.random_small(grid, 2)
    bands = o.assemble(grid, w["kappa"], I.BC_Z_DIRICHLET)
    A = D.dense_A(grid, bands)
    cz = bands[3]
    m = (nz - 1) // 2
    Pb = [A[i * nxy:(i + 1) * nxy, i * nxy:(i + 1) * nxy].copy() for i in range(nz)]
    C = [np.diag(cz[i * nxy:(i + 1) * nxy]) for i in range(nz)]
    for i in range(1, m):
        Pb[i] = Pb[i] - C[i - 1] @ np.linalg.inv(Pb[i - 1]) @ C[i - 1]
    for i in range(nz - 2, m, -1):
        Pb[i] = Pb[i] - C[i] @ np.linalg.inv(Pb[i + 1]) @ C[i]
    if m > 0:
        Pb[m] = Pb[m] - C[m - 1] @ np.linalg.inv(Pb[m - 1]) @ C[m - 1]
    if m < nz - 1:
        Pb[m] = Pb[m] - C[m] @ np.linalg.inv(Pb[m + 1]) @ C[m]
    P = sla.block_diag(*Pb)
    L3 = D.twisted_lower(nz, nxy, cz)
    B = (P + L3) @ (np.eye(nx * ny * nz) + np.linalg.inv(P) @ L3.T)
    np.testing.assert_allclose(B, A, atol=1e-12 * np.abs(A).max())


# ----------------------------------------------------------------- filtering (P3, P6)

@pytest.mark.parametrize("use_t", [False, True])
def test_level2_filtering_exact(use_t):
    """Level 2 filters exactly: B_{P,i} t_i = P_i t_i for every plane, for the
    rowsum filter t = 1 (Sec. I Eq. (4)) and a random positive t (P3)."""
    grid = (6, 5, 4)
    nx, ny, nz = grid
    n, nxy = nx * ny * nz, nx * ny
    t = np.random.default_rng(1).uniform(0.5, 2.0, n) if use_t else None
    _, _, f = _case(grid, 9, t=t)
    tt = np.ones(n) if t is None else t
    for i in range(nz):
        s = slice(i * nxy, (i + 1) * nxy)
        P = D.plane_P(nx, ny, f.Pd[s], f.Px[s], f.Py[s])
        BP = D.plane_BP(nx, ny, f.Td[s], f.To[s], f.Py[s])
        np.testing.assert_allclose(BP @ tt[s], P @ tt[s], rtol=0, atol=1e-12 * np.abs(P).max())


@pytest.mark.parametrize("use_t", [False, True])
@pytest.mark.parametrize("grid", [(1, 5, 6), (5, 1, 6), (6, 5, 1), (7, 1, 1)])
def test_filtering_exact_degenerate(grid, use_t):
    """B t = A t exactly when a dimension is 1 (P6): with one plane B = B_P and
    level 2 filters exactly; with nx = 1 or ny = 1 the level-3 beta uses an
    exact inverse.  Rowsum t = 1 and a random positive t."""
    n = int(np.prod(grid))
    t = np.random.default_rng(2).uniform(0.5, 2.0, n) if use_t else np.ones(n)
    _, bands, f = _case(grid, 4, t=t if use_t else None)
    A = D.dense_A(grid, bands)
    B, _ = D.dense_B(grid, f)
    np.testing.assert_allclose(B @ t, A @ t, rtol=0, atol=1e-11 * np.abs(A).max())


@pytest.mark.parametrize("use_t", [False, True])
@pytest.mark.parametrize("grid", [(4, 5, 6), (5, 4, 3), (3, 3, 7)])
def test_level3_filtering_defect_closed_form(grid, use_t):
    """In 3-D, (B t - A t) on plane k equals C beta (P_s - B_{P,s}) B_{P,s}^{-1} w
    summed over the planes s it is eliminated from, with w = C t_k and beta =
    (B_{P,s}^{-1} w) ./ w (the beta definition of Sec. II-A under reading R1)."""
    nx, ny, nz = grid
    nxy, n = nx * ny, nx * ny * nz
    t = np.random.default_rng(3).uniform(0.5, 2.0, n) if use_t else np.ones(n)
    _, bands, f = _case(grid, 6, t=t if use_t else None)
    A = D.dense_A(grid, bands)
    B, BP = D.dense_B(grid, f)
    defect = B @ t - A @ t
    cz = bands[3]
    m = (nz - 1) // 2
    pred = np.zeros(n)
    for k in range(nz):
        srcs = []
        if 0 < k <= m: srcs.append(k - 1)
        if m <= k < nz - 1: srcs.append(k + 1)
        for s in srcs:
            c = cz[min(s, k) * nxy:(min(s, k) + 1) * nxy]
            sl = slice(s * nxy, (s + 1) * nxy)
            Ps = D.plane_P(nx, ny, f.Pd[sl], f.Px[sl], f.Py[sl])
            BPs = BP[sl, sl]
            wv = c * t[k * nxy:(k + 1) * nxy]
            v = np.linalg.solve(BPs, wv)
            beta = v / wv
            pred[k * nxy:(k + 1) * nxy] += c * beta * ((Ps - BPs) @ v)
    assert np.linalg.norm(defect) > 1e-8 * np.linalg.norm(A @ t)     # really nonzero in 3-D
    np.testing.assert_allclose(defect, pred, rtol=0, atol=1e-10 * np.abs(A @ t).max())


# ----------------------------------------------------------------- PCG (P9, P10)

def test_pcg_monotone_A_norm_error_and_true_residual():
    """PCG (Sec. III conventions): the A-norm error decreases monotonically and
    the final true residual is below rtol (P9)."""
    grid = (6, 5, 7)
    w, bands, f = _case(grid, 8)
    A = D.dense_A(grid, bands)
    xs = np.linalg.solve(A, w["b"])
    errs = []
    for k in range(1, 12):
        r = o.pcg(grid, bands, f, w["b"], rtol=1e-300, maxit=k)
        e = r["x"] - xs
        errs.append(np.sqrt(e @ A @ e))
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1))
    res = o.pcg(grid, bands, f, w["b"], rtol=1e-8)
    assert res["status"] == 0 and res["relres"] < 1e-8
    np.testing.assert_allclose(res["x"], xs, rtol=1e-6 * np.linalg.cond(A) ** 0.5)


def test_pcg_flexible_matches_standard_for_exact_apply():
    """With an exact (FP64, fixed) preconditioner, flexible CG's beta equals the
    standard one in exact arithmetic, so both converge alike."""
    grid = (5, 5, 5)
    w, bands, f = _case(grid, 12)
    a = o.pcg(grid, bands, f, w["b"], rtol=1e-9)
    b = o.pcg(grid, bands, f, w["b"], rtol=1e-9, flexible=True)
    assert abs(a["iters"] - b["iters"]) <= 1
    np.testing.assert_allclose(a["x"], b["x"], rtol=1e-6)


def test_pcg_zero_rhs():
    grid = (3, 3, 3)
    _, bands, f = _case(grid, 1)
    res = o.pcg(grid, bands, f, np.zeros(27))
    assert res["iters"] == 0 and np.all(res["x"] == 0)


def test_lanczos_extremes_match_generalized_eigs():
    """Extreme Ritz values from the PCG coefficients approach the extreme
    eigenvalues of the pencil (A, B) (P10)."""
    grid = (5, 4, 6)
    w, bands, f = _case(grid, 13, contrast=2)
    n = int(np.prod(grid))
    A = D.dense_A(grid, bands)
    B, _ = D.dense_B(grid, f)
    ev = sla.eigh(A, 0.5 * (B + B.T), eigvals_only=True)
    res = o.pcg(grid, bands, f, w["b"], rtol=1e-14, maxit=n)
    lmin, lmax = o.lanczos_extremes(res["alpha"], res["beta"])
    assert abs(lmax - ev[-1]) <= 1e-2 * ev[-1]
    assert abs(lmin - ev[0]) <= 1e-2 * ev[0]


def test_setup_rejects_nonpositive_filter():
    grid = (3, 3, 3)
    w = I.random_small(grid, 1)
    bands = o.assemble(grid, w["kappa"], I.BC_Z_DIRICHLET)
    t = np.ones(27)
    t[5] = 0.0
    with pytest.raises(o.OracleError):
        o.setup(grid, bands, t)


# ----------------------------------------------------------------- ILU(0) smoother and B_c (Sec. III)

def _dense_ilu0(A, split):
    """Textbook ILU(0) (IKJ variant restricted to the pattern of blkD(A))."""
    n = A.shape[0]
    Ab = A.copy()
    Ab[:split, split:] = 0
    Ab[split:, :split] = 0
    pat = Ab != 0
    LU = Ab.copy()
    for i in range(1, n):
        for k in range(i):
            if pat[i, k]:
                LU[i, k] /= LU[k, k]
                js = np.nonzero(pat[i, k + 1:])[0] + k + 1
                LU[i, js] -= LU[i, k] * LU[k, js]
    return (np.tril(LU, -1) + np.eye(n)) @ np.triu(LU)


@pytest.mark.parametrize("grid", [(3, 4, 5), (4, 3, 3), (5, 1, 4), (1, 1, 6), (3, 3, 1)])
def test_ilu0_equals_textbook_ilu0_of_blkD(grid):
    """ILU(0) of blkD(A), M = floor(N/2) (Sec. III): the oracle's pivots give
    (D + L) D^{-1} (D + U) = the product of a textbook IKJ ILU(0), and the
    oracle's sweeps solve with it."""
    n = int(np.prod(grid))
    w, bands, _ = _case(grid, 21)
    A = D.dense_A(grid, bands)
    Dp = o.ilu0_setup(grid, bands)
    Bt = _dense_ilu0(A, n // 2)
    Ab = A.copy()
    Ab[: n // 2, n // 2:] = 0
    Ab[n // 2:, : n // 2] = 0
    L = np.tril(Ab, -1)
    Bo = (np.diag(Dp) + L) @ np.diag(1.0 / Dp) @ (np.diag(Dp) + L.T)
    np.testing.assert_allclose(Bo, Bt, atol=1e-12 * np.abs(A).max())
    r = np.random.default_rng(22).standard_normal(n)
    np.testing.assert_allclose(o.ilu0_solve(grid, bands, Dp, r), np.linalg.solve(Bt, r),
                               rtol=1e-10, atol=1e-12 * np.abs(np.linalg.solve(Bt, r)).max())


@pytest.mark.parametrize("grid", [(4, 5, 3), (3, 3, 3)])
def test_combination_equals_formula(grid):
    """B_c^{-1} = B_NTD^{-1} + B_ILU0^{-1} - B_NTD^{-1} A B_ILU0^{-1} (Sec. III Eq. (com))."""
    n = int(np.prod(grid))
    w, bands, f = _case(grid, 23)
    A = D.dense_A(grid, bands)
    Dp = o.ilu0_setup(grid, bands)
    Bn = np.linalg.inv(D.dense_B(grid, f)[0])
    Bi = np.linalg.inv(_dense_ilu0(A, n // 2))
    Bc = Bn + Bi - Bn @ A @ Bi
    r = np.random.default_rng(24).standard_normal(n)
    np.testing.assert_allclose(o.combo_apply(grid, bands, f, Dp, r), Bc @ r, rtol=1e-10,
                               atol=1e-12 * np.abs(Bc @ r).max())


def test_combination_error_propagator_is_product():
    """I - B_c^{-1} A = (I - B_NTD^{-1} A)(I - B_ILU0^{-1} A): the smoother and
    the NTD sweep act one after the other on the error."""
    grid = (4, 4, 5)
    n = int(np.prod(grid))
    w, bands, f = _case(grid, 25)
    A = D.dense_A(grid, bands)
    Dp = o.ilu0_setup(grid, bands)
    cols = np.column_stack([o.combo_apply(grid, bands, f, Dp, A[:, j]) for j in range(n)])
    Bn = np.linalg.inv(D.dense_B(grid, f)[0])
    Bi = np.linalg.inv(_dense_ilu0(A, n // 2))
    E = (np.eye(n) - Bn @ A) @ (np.eye(n) - Bi @ A)
    np.testing.assert_allclose(np.eye(n) - cols, E, atol=1e-9)


def test_combination_pcg_converges_fast_on_blocks32():
    """With B_c, CG on the 32^3 10^6-contrast block workload converges in a few
    dozen iterations (Table I reports 16-26 at 10^6-4.3*10^7 unknowns)."""
    w = I.workload_blocks32(seed=0)
    g = w["grid"]
    bands = o.assemble(g, w["kappa"], w["bc"])
    res = o.pcg(g, bands, o.setup(g, bands), w["b"], rtol=1e-8, maxit=200, flexible=True,
                ilu=o.ilu0_setup(g, bands))
    assert res["status"] == 0 and res["iters"] < 60 and res["relres"] < 1e-8
