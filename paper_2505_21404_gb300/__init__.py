"""GB300-native (sm_103a) Dual Natural Gradient Descent step.

The compute path lives in the CUDA library ``libdngd.so`` (C ABI in
``include/dngd.h``); ``paper_2505_21404_gb300.dngd`` is its ctypes binding and
``paper_2505_21404_gb300.workloads`` draws the seeded synthetic inputs.
Importing this package does not load the library; importing ``.dngd`` does,
and fails loudly if it has not been built.
"""
__all__ = ["dngd", "workloads"]
