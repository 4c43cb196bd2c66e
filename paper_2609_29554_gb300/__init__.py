"""GB300-native Ozaki-scheme-II multiple-precision GEMM and LU (sm_103a).

The compute path is libozlu.so (csrc/, C ABI in include/ozlu.h); the module
ozlu is its Python binding.  build.build() compiles the library in-tree.
"""
__all__ = ["ozlu", "build"]
