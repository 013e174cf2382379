"""Host-side pieces of bench.py that need no GPU."""
import numpy as np

import bench
from paper_2505_21404_gb300 import workloads


def test_sub_workload_takes_leading_points_of_each_class():
    wl = workloads.poisson_sine(5, [5, 8, 8, 1], 40, 12, k=1, seed=3, lam=1e-5)
    sub = bench._sub_workload(wl, 5)
    assert [c["count"] for c in sub["classes"]] == [5, 5]
    assert np.array_equal(sub["X"][:5], wl["X"][:5])
    assert np.array_equal(sub["X"][5:], wl["X"][40:45])
    assert np.array_equal(sub["target"][5:], wl["target"][40:45])
    # the network, parameters and class constants are those of the workload
    assert sub["widths"] == wl["widths"] and np.array_equal(sub["theta"], wl["theta"])
    assert sub["classes"][1]["c_val"] == wl["classes"][1]["c_val"]
    # the original is left as it was
    assert [c["count"] for c in wl["classes"]] == [40, 12]


def test_sub_workload_caps_at_class_size():
    wl = workloads.poisson_sine(2, [2, 4, 1], 3, 7, k=1, seed=1, lam=1e-5)
    sub = bench._sub_workload(wl, 5)
    assert [c["count"] for c in sub["classes"]] == [3, 5]
    assert sub["X"].shape == (8, 2)


def test_regime_grid_cells():
    """The regime map's default grid spans both sides of n = m (n = w^2 + 5w + 1
    for the 2-w-w-1 MLP of a 2-D input), and a command-line subset is parsed
    as given."""
    import pytest
    grid = bench._regime_grid()
    assert len(grid) == 12
    ns = {w: w * w + 5 * w + 1 for _, w in grid}
    assert ns == {15: 301, 51: 2857, 71: 5397}
    for w, n in ns.items():
        d = len(workloads.poisson_sine(2, [2, w, w, 1], 8, 2, k=2, seed=0, lam=1e-5)["theta"])
        assert d == n
    assert any(ns[w] < m for m, w in grid) and any(ns[w] > m for m, w in grid)
    assert bench._regime_grid("6300:15,300:71") == [(6300, 15), (300, 71)]
    with pytest.raises(ValueError):
        bench._regime_grid("4:15")


def test_regime_cpu_baseline_is_the_oracle():
    """The regime map's host baseline times the FP64 oracle (a tiny cell)."""
    cpu = bench._regime_cpu_baseline(m=60, w=4, seconds=0.1)
    assert cpu["kind"] == "oracle" and cpu["unit"] == "steps/s" and cpu["value"] > 0
    assert "n = 37" in cpu["sample"]          # 2-4-4-1 MLP: 4^2 + 5*4 + 1 parameters
