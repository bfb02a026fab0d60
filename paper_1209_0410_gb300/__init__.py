"""GB300-native Hypercurves: batched approximate kNN over Hilbert-curve
subindexes (arXiv:1209.0410), as CUDA kernels for sm_103a behind a C ABI.

`hc` is the binding to libhc.so (include/hc.h); `datagen` draws the seeded
synthetic inputs.
"""
