"""GB300-native LDG multigrid hot path (arXiv 2412.12506): Python binding.

The compute lives in the C-ABI library ``libldgmg.so`` (CUDA for sm_103a).
Importing this package does not load it; ``paper_2412_12506_gb300.ldgmg``
does, and raises if the library is missing.
"""
