"""GB300-native space-time multilevel Monte Carlo for the stochastic monodomain
equation (arXiv:1911.06066).

The computation is the CUDA library built from ``csrc/`` (C ABI in
``include/mlmc.h``); ``binding`` marshals arguments to it and ``workloads``
holds the synthetic benchmark configurations.  Importing this package loads
nothing; the library is loaded on first use and its absence is an error.
"""
__all__ = ["binding", "workloads", "build"]
