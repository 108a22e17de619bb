"""GB300-native mixed-precision one-sided Jacobi SVD (arXiv 2209.04626).

The compute path is the C-ABI library ``libmpjsvd.so`` (hand-written sm_103a CUDA);
``paper_2209_04626_gb300.mpjsvd`` is its thin Python binding. Importing this package
does not load the library; the binding loads it on first use and raises if it is
missing.
"""
