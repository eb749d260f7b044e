"""GB300-native hot path of a two-stage hierarchical matched-filter search.

``mf`` is the ctypes binding of libmf.so (CUDA kernels + C ABI, include/mf.h);
``hierarchy`` drives the two stages through it.  Importing the package does not
load the library; ``mf.load()`` does, and fails loudly when it is missing.
"""
