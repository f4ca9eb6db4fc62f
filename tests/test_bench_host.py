"""Host-side plumbing of bench.py (no GPU): workload names, descriptions and
the paper's test problems as bench workloads."""
import bench
import numpy as np
import pytest


@pytest.mark.parametrize("kind", [1, 2, 3])
def test_paper_workloads(kind):
    w = bench.make_workload(f"paper{kind}_12")
    assert w["grid"] == (12, 12, 12) and w["bc"] == (0, 0, 0, 0, 0, 0)
    assert w["kappa"].shape == (12 ** 3,) and np.all(w["kappa"] >= 1.0)
    assert np.allclose(w["b"], 12.0 ** -3)
    d = bench.describe(f"paper{kind}_350")
    assert f"type {kind}" in d and "350^3" in d and "Dirichlet on all faces" in d


def test_named_workloads_and_unknown_name():
    assert bench.make_workload("blocks32")["grid"] == (32, 32, 32)
    assert "350^3" in bench.describe("grf350")
    with pytest.raises(ValueError):
        bench.make_workload("nosuchworkload")


def test_reference_iterations_known_for_the_bench_workloads():
    # the reference arm extrapolates the oracle to these counts
    assert set(bench.REFERENCE_ITERS) >= {"grf350", "batched"}
    assert bench.RTOL == 1e-8
