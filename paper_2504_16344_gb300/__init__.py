"""GB300 online Bayesian inversion (arXiv 2504.16344, Phase 4) -- package.

`build` compiles libtw.so in-tree; `tw` is the ctypes binding of its C ABI
(include/tw.h).  Importing the package loads nothing on the GPU.
"""
