"""GB300-native range-mapped data-parallel kernels with energy metering.

The compute path is libsy.so (hand-written sm_103a CUDA behind a C ABI, declared
in include/sy.h); this package is its thin Python binding.  The library is
loaded on first use, not at import, so `paper_2505_06022_gb300.inputs` can be
imported on hosts without the built library.
"""
