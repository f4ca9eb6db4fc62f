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


def test_oracle_iteration_counts_stored_for_the_bench_workloads():
    """The CPU baseline and the reference arm extrapolate the oracle's time per
    iteration to the oracle's own iteration count, written by
    oracle/reference_iterations.py (never the GPU's count)."""
    for name in ("grf350", "blocks32", "batched"):
        it = bench.oracle_iterations(name)
        assert it is not None and it > 0, name
    assert bench.oracle_iterations("nosuchworkload") is None
    assert bench.RTOL == 1e-8
