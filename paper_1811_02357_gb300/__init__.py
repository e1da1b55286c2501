"""GB300-native IRT-PS (Iterative Ray Tracing Photometric Stereo).

The compute path is the CUDA library built from `csrc/` (sm_103a) behind the C
ABI in `include/irtps.h`; `irtps` is its Python binding.  Import the binding
explicitly (`from paper_1811_02357_gb300 import irtps`): it loads the library and
fails loudly if it has not been built.
"""
__all__ = ["irtps", "build"]
