"""GB300-native HOOI hot path for sparse Tucker decomposition (arXiv:1804.09494).

The compute path is the CUDA library ``libtucker.so`` (C ABI in include/tucker.h);
``tucker`` is its Python binding and ``synth`` draws seeded synthetic inputs.
"""
__all__ = ["tucker", "synth", "build"]
