"""GB300-native (sm_103a) monodomain IMEX step of lifex-ep (arXiv 2308.01651).

The compute path lives in the CUDA shared library built from ``csrc/`` and is
reached through the C ABI in ``include/ep.h``; ``ep`` is its Python binding.
``inputs`` generates the seeded synthetic workloads.
"""
