"""GB300-native incremental concatenated-matrix SVD (arXiv 2601.11626).

The compute path is the C-ABI CUDA library ``libcsvd.so`` built from
``csrc/``; ``csvd`` is its thin ctypes binding.  Importing the package does
not load the library; ``csvd.lib()`` does, and fails loudly when it is
missing.
"""
