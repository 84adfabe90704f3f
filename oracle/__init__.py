"""FP64 CPU oracle for the concatenated-matrix SVD method (arXiv 2601.11626).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of what the method computes, in float64 numpy, written from the
paper.  It shares no code with the CUDA library and is never called by the
product path: only the test-suite, the smoke check and the benchmark's CPU
baseline leg import it.

Modules
-------
exact        singular values / Eckart-Young tail of the concatenation
             (Problem Formulation; Thm. 4 Eckart-Young-Mirsky, Appendix A),
             exact tail gradient.
incremental  the incremental truncated-SVD estimator (Lemma 1 and Cor. 3 of
             Appendix B) and the plug-in tail estimate (Cor. 2, Section 3.3).
bounds       Weyl-type bound (Thm. 1) and residual bound (Thm. 2, Cor. 1).
cluster      Algorithms 1-3 of Appendix E and the compression ratio (Section 4).
decomp       the final per-cluster decomposition and its true error.
stream       streaming cluster assignment (the discussion section's
             incremental setting).
randomized   the randomized range-finder tail estimate (the discussion
             section's sketching variant), certified by its explicit residual.

Every reading of a passage that is silent or ambiguous is listed in the
module that applies it (look for "Reading").
"""
from . import exact, incremental, bounds, cluster, randomized  # noqa: F401
