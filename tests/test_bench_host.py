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
