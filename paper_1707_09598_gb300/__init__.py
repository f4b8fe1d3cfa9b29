"""GB300-native sparse-grid isogeometric Poisson solver (arXiv:1707.09598).

The compute path is the CUDA library libsgiga.so (csrc/, C ABI in
include/sgiga.h); `sgiga` is its Python binding and `build` compiles it.
"""
