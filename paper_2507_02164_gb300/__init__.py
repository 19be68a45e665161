"""GB300-native batched complex polynomial roots and root-density histograms.

Method: Tang & Quan, "Hardware-Accelerated Algorithm for Complex Function
Roots Density Graph Plotting" (arXiv 2507.02164). The compute path is the
CUDA library libroots (C ABI in include/rootdensity.h); ``api`` binds it over
torch tensors, ``workloads`` holds the seeded synthetic inputs.
"""
__all__ = ["api", "workloads", "build"]
