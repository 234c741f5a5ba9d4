"""GB300-native relaxing-TVD patch-group hydro path of GAMER (arXiv 0907.3390).

The compute path lives in ``libgamer_hydro.so`` (hand-written CUDA for
sm_103a behind a C ABI, declared in ``include/gamer_hydro.h``); ``binding``
marshals arguments to it.  ``hierarchy`` and ``workloads`` build neighbour
maps and seeded synthetic inputs on the host.  Importing this package does
not load the CUDA library; ``binding.load()`` does, and fails loudly if it
is missing.
"""
__all__ = ["hierarchy", "workloads", "binding"]
