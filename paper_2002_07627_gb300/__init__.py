"""GB300-native inaccessibility measure field (IMF) library, arXiv 2002.07627.

The computation lives in the CUDA library libimf (csrc/, C ABI in include/imf.h); `binding`
is a thin ctypes layer over it, `synth` builds seeded synthetic inputs, `build` compiles the
library in-tree for sm_103a. Importing this package loads nothing: the library is loaded on
first use and a missing build raises instead of falling back to any CPU path.
"""
__all__ = ["binding", "build", "synth"]
