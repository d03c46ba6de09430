"""GB300-native pseudo-Verlet SPH density loop (arXiv:1804.06231 hot path).

``inputs`` draws seeded synthetic particle sets.  The CUDA library and its
binding are loaded by ``paper_1804_06231_gb300.pv`` on first use.
"""
__all__ = ["inputs"]
