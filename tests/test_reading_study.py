"""Pins of the two Schur-term forms of the oracle against the independent dense
construction of tests/reading_study.py, and the study's findings on small
grids (CPU only).

Sec. II-A prints the approximate inverse X = 2 beta - beta P beta for the
Schur terms of both the plane and the line recurrences, and calls it a better
approximation than beta itself; the oracle and the library implement it, and
also X = beta (FFP_SCHUR_BETA).  The dense construction is written from the
definitions alone (twisted block recurrences, B = (B_P + L3) B_P^{-1}
(B_P + U3), B_P = (T + L2) T^{-1} (T + U2)) and shares no code with the
oracle; the oracle's apply must equal its B^{-1} for either form.
"""
import numpy as np
import pytest

from oracle import oracle as o
from paper_1909_09771_gb300 import inputs as I
from tests import reading_study as RS


def _relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("schur", ["newton", "beta"])
@pytest.mark.parametrize("grid", [(5, 6, 7), (3, 8, 2), (4, 4, 4), (6, 1, 5), (1, 5, 4), (2, 2, 3), (7, 3, 1)])
def test_oracle_apply_equals_dense_construction(grid, schur):
    w = I.random_small(grid, 21, contrast_exp=3)
    bands = o.assemble(grid, w["kappa"], w["bc"])
    B, _, _ = RS.dense_ntd(grid, bands, schur, schur, "nested")
    r = np.random.default_rng(22).standard_normal(int(np.prod(grid)))
    z = o.apply(o.setup(grid, bands, schur=schur), r)
    assert _relerr(z, np.linalg.solve(B, r)) <= 1e-11


def test_exact_schur_terms_give_A():
    """With the exact inverse at level 3 (no level-2 approximation), B = A
    (the twisted block LU, Sec. II-A): the construction's bookkeeping check."""
    grid = (4, 3, 5)
    w = I.random_small(grid, 23, contrast_exp=2)
    bands = o.assemble(grid, w["kappa"], w["bc"])
    B, _, _ = RS.dense_ntd(grid, bands, "exact", "newton", "exact")
    A = RS.D.dense_A(grid, bands)
    assert np.max(np.abs(B - A)) <= 1e-10 * np.max(np.abs(A))


def test_beta_form_keeps_filtering_property():
    """X = beta satisfies X w = P^{-1} w like the printed form, so level-2
    filtering B_P t = P t holds plane by plane (rowsum t = 1)."""
    grid = (6, 5, 4)
    w = I.random_small(grid, 24, contrast_exp=3)
    bands = o.assemble(grid, w["kappa"], w["bc"])
    f = o.setup(grid, bands, schur="beta")
    nx, ny, nz = grid
    for i in range(nz):
        s = slice(i * nx * ny, (i + 1) * nx * ny)
        P = RS.D.plane_P(nx, ny, f.Pd[s], f.Px[s], f.Py[s])
        BP, _ = RS.plane_bp(P, nx, ny, "beta")
        t = np.ones(nx * ny)
        assert _relerr(BP @ t, P @ t) <= 1e-12


def test_study_findings_grf8():
    """The study's finding on the 10^6-contrast GRF at 8^3: the inverse inside
    beta-hat (nested solve of reading R1, or the exact inverse) changes the
    B_NTD iteration count by under 5 %; the printed X is strongly indefinite
    at both levels and B_NTD needs over 500 iterations, while X = beta keeps
    lambda(B^{-1} A) in [0.99, 3] and needs under 20."""
    w = I.workload_grf(seed=0, n=8)
    bands = o.assemble(w["grid"], w["kappa"], w["bc"])
    rows = {r[1]: r for r in RS.study("grf8", w["grid"], bands,
                                         [("newton", "newton", "nested"), ("newton", "newton", "exact"),
                                          ("beta", "beta", "nested")])}
    nn, ne, bb = rows[("newton", "newton", "nested")], rows[("newton", "newton", "exact")], rows[("beta", "beta", "nested")]
    assert abs(nn[6] - ne[6]) <= 0.05 * nn[6]
    assert nn[4] < -1.0 and nn[5] < -1.0          # negative eigenvalues dominate X at both levels
    assert nn[6] > 500
    assert 0.99 <= bb[2] and bb[3] <= 3.0 and bb[6] < 20
