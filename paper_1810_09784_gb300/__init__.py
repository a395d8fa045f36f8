"""Generalized FrequencyHough (Miller et al., arXiv:1810.09784) for GB300.

`gfh` is the binding of the CUDA library libgfh (include/gfh.h); `synth` draws seeded synthetic
inputs; `workloads` holds the sizes of the synthetic searches; `build` compiles the library.
"""
