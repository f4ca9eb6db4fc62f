"""The paper's test problems (Sec. IV, "Test Matrices") as inputs: the kappa
generators checked cell by cell against values worked out by hand from the
definitions, and the Table I fixture (tests/golden/paper_table1.txt)."""
import os

import numpy as np

from paper_1909_09771_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_table1.txt")


def load_table1():
    rows = {}
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            kind, n, tol, setup, solve, overall, iters = line.split()
            rows[(int(kind), int(n), float(tol))] = dict(setup_s=float(setup), solve_s=float(solve),
                                                        overall_s=float(overall), iters=int(iters))
    return rows


def at(k, n, x, y, z):
    return k[x + n * (y + n * z)]


def test_table1_fixture():
    t = load_table1()
    assert len(t) == 18
    for kind in (1, 2, 3):
        for tol in (1e-7, 1e-10):
            its = [t[(kind, n, tol)]["iters"] for n in (100, 200, 350)]
            assert its == sorted(its)  # more iterations on finer grids
            for n in (100, 200, 350):
                r = t[(kind, n, tol)]
                assert abs(r["setup_s"] + r["solve_s"] - r["overall_s"]) <= 0.02


def test_type1_skyscrapers():
    n = 100
    k = I.kappa_paper(1, n)
    # cell centre ((x + 1/2)/n, ...): integer parts of 10 x_i for x, y, z = 5, 25, 45 are 0, 2, 4
    assert at(k, n, 5, 25, 45) == 1e3 * (2 + 1)
    assert at(k, n, 15, 25, 45) == 1.0      # [10 x_1] = 1 is odd
    assert at(k, n, 5, 85, 5) == 1e3 * (8 + 1)
    assert at(k, n, 5, 95, 5) == 1.0        # [10 x_2] = 9 is odd
    assert at(k, n, 99, 0, 99) == 1.0       # [10 x_1] = 9
    assert at(k, n, 80, 40, 0) == 1e3 * (4 + 1)
    assert sorted(set(k.tolist())) == [1.0, 1e3, 3e3, 5e3, 7e3, 9e3]
    assert np.count_nonzero(k > 1) * 8 == n ** 3  # the even blocks are 1/8 of the cube


def test_type2_ring():
    n = 100
    k = I.kappa_paper(2, n)
    assert at(k, n, 50, 50, 50) == 1.0      # centre, |x - c| = 0.0087
    assert at(k, n, 50, 50, 16) == 1.0      # |x - c| = 0.3351 < 1/(2 sqrt 2) = 0.3536
    assert at(k, n, 50, 50, 10) == 1e3      # 0.3951
    assert at(k, n, 50, 50, 0) == 1e3       # 0.4950
    assert at(k, n, 0, 50, 50) == 1e3
    assert at(k, n, 0, 0, 50) == 1.0        # 0.7001
    # shell volume 4/3 pi (1/8 - (1/(2 sqrt 2))^3) = 0.3385 of the cube
    frac = np.count_nonzero(k > 1) / n ** 3
    assert abs(frac - 4.0 / 3.0 * np.pi * (0.125 - (0.5 / np.sqrt(2.0)) ** 3)) < 0.01


def test_type3_poisson_and_workload():
    w = I.workload_paper(3, 20)
    assert np.all(w["kappa"] == 1.0)
    assert w["bc"] == (0, 0, 0, 0, 0, 0)
    assert w["grid"] == (20, 20, 20)
    assert np.allclose(w["b"], (1.0 / 20) ** 3)
