"""GB300-native RBF semi-Lagrangian transport on the sphere (sm_103a CUDA + C ABI).

The CUDA library is loaded lazily by ``paper_1804_01609_gb300.rbfsl``; ``inputs`` holds the
seeded synthetic workload generators.
"""
__all__ = ["inputs", "rbfsl", "build"]
